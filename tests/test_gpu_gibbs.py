"""The paper's Gibbs sampler on the amplitude AC (GPU) against the plain oracle chain,
and its stationary distribution against the density-matrix oracle."""
import numpy as np
import pytest

from oracle import gibbs as G
from oracle import quantum as Q
from paper_2103_17226_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("prec", [64, 32])
def test_gibbs_trajectories_match_oracle(cuda_ctx, prec):
    from paper_2103_17226_gb300 import native as N
    c = I.random_circuit(3, 7, seed=950, noise_prob=0.5)
    n_ch = len(Q.channel_cards(c))
    V = 2
    angs = I.uniform_angles(V, c.n_angles, seed=95)
    ac = N.load_ac(cuda_ctx, N.compile(c, N.QKC_AC_AMPLITUDE), precision=prec)
    N.set_params(ac, torch.tensor(angs, device="cuda"))
    chains = 6
    seeds = I.vector_seeds(chains, 95)
    # start: outputs from the noise-free branch with the largest amplitude, every noise variable 0
    start = []
    for ch in range(chains):
        psi = Q.statevector(c, angs[ch % V], [0] * n_ch)
        x = int(np.argmax(np.abs(psi.reshape(-1))))
        start.append([(x >> (2 - q)) & 1 for q in range(3)] + [0] * n_ch)
    state = torch.tensor(np.array(start, dtype=np.int8), device="cuda")
    cv = torch.tensor([ch % V for ch in range(chains)], dtype=torch.int32, device="cuda")
    samples = N.gibbs(ac, cv, torch.tensor(seeds.astype(np.int64), device="cuda"), state, 4)
    samples = samples.cpu().numpy()
    final = state.cpu().numpy()
    mism = 0
    for ch in range(chains):
        ref_state, ref_out = G.gibbs_chain(c, angs[ch % V], start[ch], int(seeds[ch]), 4)
        mism += int(list(final[ch]) != ref_state) + int(list(samples[ch].astype(np.uint64)) != ref_out)
    assert mism <= (0 if prec == 64 else 1)


def test_gibbs_stationary_distribution(cuda_ctx):
    from scipy.stats import chisquare
    from paper_2103_17226_gb300 import native as N
    c = I.workload("qaoa4_ring_p1")
    n_ch = len(Q.channel_cards(c))
    ang = I.uniform_angles(1, c.n_angles, seed=44)
    ac = N.load_ac(cuda_ctx, N.compile(c, N.QKC_AC_AMPLITUDE), precision=32)
    N.set_params(ac, torch.tensor(ang, device="cuda"))
    chains = 4096
    psi = Q.statevector(c, ang[0], [0] * n_ch).reshape(-1)
    x0 = int(np.argmax(np.abs(psi)))
    st = np.zeros((chains, 4 + n_ch), dtype=np.int8)
    st[:, :4] = [(x0 >> (3 - q)) & 1 for q in range(4)]
    state = torch.tensor(st, device="cuda")
    cv = torch.zeros(chains, dtype=torch.int32, device="cuda")
    seeds = torch.tensor(I.vector_seeds(chains, 44).astype(np.int64), device="cuda")
    out = N.gibbs(ac, cv, seeds, state, 40).cpu().numpy()
    last = out[:, -1]  # one draw per chain after 39 burn-in sweeps
    P = Q.probabilities(c, ang[0])
    counts = np.bincount(last, minlength=16).astype(float)
    keep = P * chains > 5
    exp = P[keep] * chains
    obs = counts[keep] * exp.sum() / counts[keep].sum()
    assert chisquare(obs, exp).pvalue > 0.01
