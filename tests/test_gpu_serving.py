"""Serving loop (GPU): continuous batching over resident ACs gives every request the same
samples alone and in the mix; the FP64 one-request-at-a-time path matches the oracle."""
import numpy as np
import pytest

from oracle import quantum as Q
from paper_2103_17226_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _acs(kind=1):
    from paper_2103_17226_gb300 import native as N
    circs = {
        "qaoa6": I.qaoa_maxcut(6, I.random_regular_graph(6, 3, 61), 1, I.NOISE_CFG2, name="qaoa6"),
        "qaoa8": I.qaoa_maxcut(8, I.random_regular_graph(8, 3, 81), 1, I.NOISE_CFG2, name="qaoa8"),
        "hea4": I.hardware_efficient_ansatz(4, 2, I.NOISE_CFG3, name="hea4"),
    }
    return circs, {k: N.compile(c, kind) for k, c in circs.items()}


@pytest.mark.parametrize("kind", [1, 2])
def test_alone_equals_mix_and_fp64_matches_oracle(cuda_ctx, kind):
    """kind 1: density ACs; kind 2: light-cone step ACs (what the serving bench keeps resident)."""
    from paper_2103_17226_gb300.serve import Request, Server, poisson_requests
    circs, acs = _acs(kind)
    n_angles = {k: c.n_angles for k, c in circs.items()}
    reqs = poisson_requests(list(acs), n_angles, rate_per_s=20000.0, duration_s=0.004, seed=7, shots_lo=50,
                            shots_hi=1500)
    assert len(reqs) >= 40
    srv = Server(cuda_ctx, acs, precision=32, lanes=2, max_batch=8, max_shots=1500, tile_columns=2048)
    res, stats = srv.run(reqs)
    assert stats["completed"] == len(reqs)
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    # alone: a serial server with batches of one request
    alone = Server(cuda_ctx, acs, precision=32, lanes=1, max_batch=1, max_shots=1500, tile_columns=2048,
                   serial=True)
    pick = reqs[::5]
    res1, _ = alone.run([Request(r.rid, r.ac, r.angles, r.shots, r.seed, 0.0) for r in pick])
    for r in pick:
        assert np.array_equal(res1[r.rid].bits, res[r.rid].bits), r.rid
    # the FP64 one-request-at-a-time path against the oracle's chain rule
    base = Server(cuda_ctx, acs, precision=64, lanes=1, max_batch=1, max_shots=1500, tile_columns=2048,
                  serial=True)
    few = [r for r in reqs if r.ac in ("qaoa6", "hea4")][:6]
    res64, _ = base.run([Request(r.rid, r.ac, r.angles, r.shots, r.seed, 0.0) for r in few])
    mism = 0
    for r in few:
        P = Q.probabilities(circs[r.ac], r.angles)
        ref = Q.chain_rule_samples(P, r.seed, r.shots)
        mism += int((res64[r.rid].bits.astype(np.uint64) != ref).sum())
    assert mism == 0


def test_mix_with_trajectory_ac_and_refused_requests(cuda_ctx):
    """A TRAJECTORY AC (mixed-unitary noise, p=2) resident beside density ACs: its requests give the same
    samples alone and in the mix, the FP64 one-request path matches the trajectory oracle, and a request
    with more shots than a lane holds is refused and counted, not served."""
    from oracle import trajectory as T
    from paper_2103_17226_gb300 import native as N
    from paper_2103_17226_gb300.serve import Request, Server, poisson_requests
    circs, acs = _acs(1)
    circs["qaoa6_p2"] = I.qaoa_maxcut(6, I.random_regular_graph(6, 3, 62), 2, I.NOISE_CFG2, name="qaoa6_p2")
    acs["qaoa6_p2"] = N.compile(circs["qaoa6_p2"], N.QKC_AC_TRAJECTORY)
    n_angles = {k: c.n_angles for k, c in circs.items()}
    reqs = poisson_requests(list(acs), n_angles, rate_per_s=20000.0, duration_s=0.004, seed=9, shots_lo=50,
                            shots_hi=1500)
    big = Request(10 ** 6, "qaoa6_p2", np.zeros(n_angles["qaoa6_p2"]), 2000, 5, 0.0)  # more shots than a lane holds
    srv = Server(cuda_ctx, acs, precision=32, lanes=2, max_batch=8, max_shots=1500, tile_columns=2048)
    res, stats = srv.run(reqs + [big])
    assert stats["completed"] == len(reqs) and stats["refused"] == 1 and big.rid not in res
    assert stats["unfinished"] == 0
    traj = [r for r in reqs if r.ac == "qaoa6_p2"]
    assert len(traj) >= 5
    alone = Server(cuda_ctx, acs, precision=32, lanes=1, max_batch=1, max_shots=1500, tile_columns=2048,
                   serial=True)
    res1, _ = alone.run([Request(r.rid, r.ac, r.angles, r.shots, r.seed, 0.0) for r in traj[:5]])
    for r in traj[:5]:
        assert np.array_equal(res1[r.rid].bits, res[r.rid].bits), r.rid
    base = Server(cuda_ctx, acs, precision=64, lanes=1, max_batch=1, max_shots=1500, tile_columns=2048,
                  serial=True)
    res64, _ = base.run([Request(r.rid, r.ac, r.angles, r.shots, r.seed, 0.0) for r in traj[:3]])
    for r in traj[:3]:
        want = T.trajectory_samples(circs["qaoa6_p2"], r.angles, r.seed, r.shots)
        assert np.array_equal(res64[r.rid].bits.astype(np.uint64), want), r.rid
