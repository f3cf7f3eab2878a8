"""ACExpectation: the autograd wrapper's forward and backward against the oracle (GPU)."""
import numpy as np
import pytest

from oracle import quantum as Q
from paper_2103_17226_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("prec", [64, 32])
def test_expectation_forward_backward(cuda_ctx, prec):
    from paper_2103_17226_gb300 import native as N
    from paper_2103_17226_gb300.torch_ops import expectation, z_string_columns
    c = I.hardware_efficient_ansatz(4, 2, I.NOISE_CFG3)
    V = 3
    sup, coef = I.z_string_hamiltonian(4, 5, seed=41)
    ac = N.load_ac(cuda_ctx, N.compile(c, N.QKC_AC_DENSITY), precision=prec)
    ang0 = I.uniform_angles(V, c.n_angles, seed=41)
    angles = torch.tensor(ang0, device="cuda", requires_grad=True)
    cv, ev, w = z_string_columns(sup, coef, V, 4)
    val = expectation(angles, ac, cv, ev, w)
    upstream = torch.tensor([1.0, -2.0, 0.5], device="cuda", dtype=torch.float64)
    (val * upstream).sum().backward()
    tol = (1e-12 if prec == 64 else 1e-5) * np.abs(coef).sum()
    for v in range(V):
        rv, rg = Q.hamiltonian_value_and_gradient(c, ang0[v], sup, coef)
        assert abs(val[v].item() - rv) < tol
        assert np.abs(angles.grad[v].cpu().numpy() - upstream[v].item() * rg).max() < 10 * tol * abs(upstream[v].item())


def test_gradient_descent_lowers_energy(cuda_ctx):
    from paper_2103_17226_gb300 import native as N
    from paper_2103_17226_gb300.torch_ops import expectation, z_string_columns
    c = I.hardware_efficient_ansatz(4, 2, I.NOISE_CFG3)
    sup, coef = I.z_string_hamiltonian(4, 5, seed=42)
    ac = N.load_ac(cuda_ctx, N.compile(c, N.QKC_AC_DENSITY), precision=32)
    angles = torch.tensor(I.uniform_angles(1, c.n_angles, seed=42), device="cuda", requires_grad=True)
    cv, ev, w = z_string_columns(sup, coef, 1, 4)
    opt = torch.optim.SGD([angles], lr=0.1)
    first = None
    for _ in range(30):
        opt.zero_grad()
        e = expectation(angles, ac, cv, ev, w).sum()
        first = e.item() if first is None else first
        e.backward()
        opt.step()
    final = expectation(angles, ac, cv, ev, w).sum().item()
    assert final < first - 0.05
    # and the final energy agrees with the density-matrix oracle
    P = Q.probabilities(c, angles.detach().cpu().numpy()[0])
    assert abs(final - sum(cf * Q.z_expectation(P, s) for s, cf in zip(sup, coef))) < 1e-5 * np.abs(coef).sum()
