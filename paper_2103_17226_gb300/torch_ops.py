"""PyTorch autograd wrapper: the expectation of a Z-string Hamiltonian, differentiable
in the gate angles, computed by the library's upward pass (value) and downward pass
(adjoints of the parameter leaves, chained with d leaf / d angle)."""
from __future__ import annotations

import torch

from . import native as N


class ACExpectation(torch.autograd.Function):
    """value[v] = sum_{c: col_vec[c] = v} weight[c] Re f(lambda_c) for each parameter vector v.

    forward(angles [V][n_angles] float64 CUDA, ac, col_vec [C] int32, evidence [C][n_vars] int8,
    weight [C] float64) -> value [V].  With one column per Z-string term (evidence code -2 on the
    term's support, -1 elsewhere) and weight = its coefficient, value is <H> per vector.  The
    gradient is computed in the same call (one upward + one downward pass per column) and
    saved for backward."""

    @staticmethod
    def forward(ctx, angles, ac, col_vec, evidence, weight):
        a = angles.detach().to(torch.float64).contiguous()
        N.set_params(ac, a)
        value, grad = N.gradient(ac, col_vec, evidence, weight, a.shape[0])
        ctx.save_for_backward(grad)
        return value

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return (g[:, None] * grad).to(g.dtype), None, None, None, None


def z_string_columns(supports, coefs, n_vectors, n_vars, device="cuda"):
    """Evidence, column map and weights for sum_t c_t Z_{S_t} over n_vectors vectors."""
    T = len(coefs)
    ev = torch.full((n_vectors * T, n_vars), -1, dtype=torch.int8)
    for t, s in enumerate(supports):
        for q, on in enumerate(s):
            if on:
                ev[t::T, q] = -2
    cv = torch.arange(n_vectors, dtype=torch.int32).repeat_interleave(T)
    w = torch.as_tensor(coefs, dtype=torch.float64).repeat(n_vectors)
    return cv.to(device), ev.to(device), w.to(device)


def expectation(angles, ac, col_vec, evidence, weight):
    return ACExpectation.apply(angles, ac, col_vec, evidence, weight)
