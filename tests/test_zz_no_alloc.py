"""qkc_evaluate_static: the upward pass for callers that cannot allocate device memory
(a latency-bound serving loop that must not stall on cudaMalloc/cudaFree, or a host
whose own pool owns the device memory).  It must give what qkc_evaluate gives, within
the tolerances of the other GPU tests, on consecutive calls that share its fixed scratch.
Collected last on purpose: it adds nothing the rest of the suite depends on."""
import ctypes

import numpy as np
import pytest

from paper_2103_17226_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = {64: 1e-12, 32: 1e-5}


def _columns(n, cols, V, seed):
    rng = I.SplitMix(seed)
    ev = np.array([[rng.randint(4) - 2 for _ in range(n)] for _ in range(cols)], dtype=np.int8)
    cv = np.array([rng.randint(V) for _ in range(cols)], dtype=np.int32)
    return torch.tensor(ev, device="cuda"), torch.tensor(cv, device="cuda")


@pytest.mark.parametrize("prec", [32, 64])
def test_static_scratch_matches_allocating_path_twice(cuda_ctx, prec):
    from paper_2103_17226_gb300 import native as N
    c = I.workload("qaoa4_ring_p1")
    V = 8
    ac = N.load_ac(cuda_ctx, N.compile(c, N.QKC_AC_DENSITY), precision=prec)
    N.set_params(ac, torch.tensor(I.uniform_angles(V, c.n_angles, seed=31), device="cuda"))
    lib = N.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # a first call: the library's module data (the fixed array among it) may be set up lazily on first use
    ev, cv = _columns(4, 64, V, 0)
    warm = torch.empty((64, 2), dtype=torch.float64, device="cuda")
    assert lib.qkc_evaluate_static(ac._h, ctypes.c_void_p(cv.data_ptr()), ctypes.c_void_p(ev.data_ptr()), 64,
                                   ctypes.c_void_p(warm.data_ptr()), stream) == 0, lib.qkc_last_error()
    # 20000 columns: several tiles of the fixed scratch; two different calls in a row
    for call, seed in enumerate((1, 2)):
        ev, cv = _columns(4, 20000, V, seed)
        want = N.evaluate(ac, cv, ev)
        got = torch.full_like(want, float("nan"))
        torch.cuda.synchronize()
        free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
        st = lib.qkc_evaluate_static(ac._h, ctypes.c_void_p(cv.data_ptr()), ctypes.c_void_p(ev.data_ptr()),
                                     ev.shape[0], ctypes.c_void_p(got.data_ptr()), stream)
        assert st == 0, lib.qkc_last_error()
        torch.cuda.synchronize()
        # the property the entry point exists for: the call allocated no device memory
        assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_reserved() == reserved0, call
        assert torch.isfinite(got).all()
        assert (got - want).abs().max().item() < TOL[prec], call


def test_static_scratch_rejects_an_ac_that_does_not_fit(cuda_ctx):
    from paper_2103_17226_gb300 import native as N
    c = I.workload("qaoa32_3reg_p1_ideal")  # ~142K nodes: more than the fixed scratch holds for 64 columns
    ac = N.load_ac(cuda_ctx, N.compile(c, N.QKC_AC_DENSITY), precision=32)
    N.set_params(ac, torch.tensor(I.uniform_angles(2, c.n_angles, seed=3), device="cuda"))
    ev = torch.full((4, 32), -1, dtype=torch.int8, device="cuda")
    cv = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.empty((4, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(N.QKCError) as e:
        N.evaluate_static(ac, cv, ev, out)
    assert e.value.status == 7 and "static scratch" in str(e.value)
