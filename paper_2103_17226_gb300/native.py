"""Thin ctypes binding of libqkc (include/qkc.h): argument marshalling only.

Every function here has the name of the C entry point without its `qkc_`
prefix and forwards to it; all computation runs in the library's CUDA kernels
(or, for `compile` and `plan`, in its host compiler).  Device buffers are
PyTorch tensors, streams are PyTorch's current stream.  There is no fallback:
if the library is missing, loading fails with an error that says so.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

from .inputs import OP_DTYPE

_LIB_PATH = Path(__file__).resolve().parent / "_build" / "libqkc.so"
_lib = None

QKC_AC_AMPLITUDE = 0
QKC_AC_DENSITY = 1
QKC_AC_DENSITY_STEPS = 2  # one density AC per sampling step (backward light cones), qkc_sample and qkc_evaluate only
QKC_AC_TRAJECTORY = 3  # doubled network with per-copy noise variables: |A(x, r)|^2 for an observed trajectory r
STATUS = {0: "QKC_OK", 1: "QKC_ERR_ARG", 2: "QKC_ERR_FORMAT", 3: "QKC_ERR_NOMEM", 4: "QKC_ERR_CUDA",
          5: "QKC_ERR_TIMEOUT", 6: "QKC_ERR_UNSUPPORTED", 7: "QKC_ERR_TOO_LARGE"}


class QKCError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class ACInfo(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n_qubits", ctypes.c_int32), ("n_angles", ctypes.c_int32),
                ("n_vars", ctypes.c_int32), ("n_ind", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("n_nodes", ctypes.c_int64), ("n_edges", ctypes.c_int64), ("n_levels", ctypes.c_int64),
                ("n_leaves", ctypes.c_int64), ("max_level_width", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("reserved_columns", ctypes.c_int64)]


class Stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("records", ctypes.c_int64),
                ("up_passes", ctypes.c_int64), ("up_columns", ctypes.c_int64), ("up_launches", ctypes.c_int64),
                ("up_ms", ctypes.c_double), ("up_bytes", ctypes.c_double),
                ("down_passes", ctypes.c_int64), ("down_columns", ctypes.c_int64), ("down_launches", ctypes.c_int64),
                ("down_ms", ctypes.c_double), ("down_bytes", ctypes.c_double),
                ("memo_passes", ctypes.c_int64), ("memo_columns", ctypes.c_int64),
                ("memo_ms", ctypes.c_double), ("memo_bytes", ctypes.c_double),
                ("memo_a_ms", ctypes.c_double), ("memo_a_bytes", ctypes.c_double),
                ("up_edges", ctypes.c_double), ("down_edges", ctypes.c_double), ("memo_edges", ctypes.c_double)]


def lib():
    """The loaded libqkc (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not _LIB_PATH.exists():
        raise RuntimeError(f"libqkc is not built ({_LIB_PATH} missing): run __graft_entry__.build() "
                           "or paper_2103_17226_gb300.build.build_library()")
    L = ctypes.CDLL(str(_LIB_PATH))
    P, I32, I64, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    sig = {
        "qkc_compile": [P, I32, I32, I32, I32, I32, I64, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(U64)],
        "qkc_plan": [P, I32, I32, I32, I32, I32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
        "qkc_ctx_create": [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)],
        "qkc_load_ac": [P, P, U64, I32, ctypes.POINTER(ctypes.c_void_p)],
        "qkc_get_info": [P, ctypes.POINTER(ACInfo)],
        "qkc_reserve": [P, I64, I64],
        "qkc_set_tile_limit": [P, I64],
        "qkc_set_params": [P, P, I64, P],
        "qkc_evaluate": [P, P, P, I64, P, P],
        "qkc_reevaluate": [P, I32, P, I64, P, P],
        "qkc_marginals": [P, P, P, I64, P, P, P],
        "qkc_gradient": [P, P, P, P, I64, I64, P, P, P],
        "qkc_sample": [P, P, P, I64, I64, I64, P, P],
        "qkc_sample_probs": [P, P, P, I64, I64, I64, P, P, P],
        "qkc_check_status": [P],
        "qkc_gibbs": [P, P, P, I64, P, I64, I64, P, P],
        "qkc_set_sampler": [P, I32, I64],
        "qkc_evaluate_static": [P, P, P, I64, P, P],
        "qkc_stats_enable": [P, I32, I64],
        "qkc_get_stats": [P, ctypes.POINTER(Stats)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.qkc_free_bytes.argtypes = [ctypes.c_void_p]
    L.qkc_free_bytes.restype = None
    L.qkc_ctx_destroy.argtypes = [ctypes.c_void_p]
    L.qkc_ctx_destroy.restype = None
    L.qkc_free_ac.argtypes = [ctypes.c_void_p]
    L.qkc_free_ac.restype = None
    L.qkc_last_error.argtypes = []
    L.qkc_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(st: int):
    if st != 0:
        raise QKCError(st, lib().qkc_last_error().decode())


def _ptr(t):
    return ctypes.c_void_p(0) if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


# --------------------------------------------------------------------------- compiler (host)
def _records(circuit):
    rec = circuit.as_records()
    assert rec.dtype == OP_DTYPE
    return np.ascontiguousarray(rec)


def compile(circuit, kind: int = QKC_AC_DENSITY, order: int = 0, max_nodes: int = 0) -> bytes:
    """qkc_compile: circuit -> compiled-AC bytes."""
    rec = _records(circuit)
    out = ctypes.c_void_p()
    n = ctypes.c_uint64()
    _check(lib().qkc_compile(rec.ctypes.data_as(ctypes.c_void_p), len(rec), circuit.n_qubits, circuit.n_angles,
                             kind, order, max_nodes, ctypes.byref(out), ctypes.byref(n)))
    try:
        return ctypes.string_at(out, n.value)
    finally:
        lib().qkc_free_bytes(out)


def plan(circuit, kind: int = QKC_AC_DENSITY, order: int = 0):
    """qkc_plan: (sum of elimination table sizes, log2 of the largest table) without building."""
    rec = _records(circuit)
    a = ctypes.c_double()
    w = ctypes.c_double()
    _check(lib().qkc_plan(rec.ctypes.data_as(ctypes.c_void_p), len(rec), circuit.n_qubits, circuit.n_angles,
                          kind, order, ctypes.byref(a), ctypes.byref(w)))
    return a.value, w.value


def header(ac_bytes: bytes) -> dict:
    """Header fields of compiled-AC bytes (the format is documented in include/qkc.h)."""
    h = np.frombuffer(ac_bytes[:64], dtype="<u4")
    keys = ["magic", "version", "kind", "n_qubits", "n_angles", "n_vars", "n_nodes", "n_edges", "n_levels",
            "n_leaves", "root", "n_ind"]
    return {k: int(h[i]) for i, k in enumerate(keys)}


# --------------------------------------------------------------------------- engine
class Context:
    """qkc_ctx_create / qkc_ctx_destroy."""

    def __init__(self, device: int = 0):
        self._h = ctypes.c_void_p()
        _check(lib().qkc_ctx_create(device, ctypes.byref(self._h)))
        self.device = device

    def close(self):
        if self._h:
            lib().qkc_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class AC:
    """A compiled AC resident on the device (qkc_load_ac / qkc_free_ac)."""

    def __init__(self, ctx: Context, ac_bytes: bytes, precision: int = 32):
        self.ctx = ctx
        self._h = ctypes.c_void_p()
        buf = ctypes.create_string_buffer(ac_bytes, len(ac_bytes))
        _check(lib().qkc_load_ac(ctx._h, buf, len(ac_bytes), precision, ctypes.byref(self._h)))
        self.precision = precision
        self._info = self.info()

    def info(self) -> dict:
        i = ACInfo()
        _check(lib().qkc_get_info(self._h, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in ACInfo._fields_}

    @property
    def n_qubits(self):
        return self._info["n_qubits"]

    @property
    def n_vars(self):
        return self._info["n_vars"]

    @property
    def n_ind(self):
        return self._info["n_ind"]

    @property
    def n_angles(self):
        return self._info["n_angles"]

    def close(self):
        if self._h:
            lib().qkc_free_ac(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ctx_create(device: int = 0) -> Context:
    return Context(device)


def load_ac(ctx: Context, ac_bytes: bytes, precision: int = 32) -> AC:
    return AC(ctx, ac_bytes, precision)


def reserve(ac: AC, max_vectors: int, max_columns: int):
    _check(lib().qkc_reserve(ac._h, max_vectors, max_columns))


def set_tile_limit(ac: AC, max_tile_columns: int):
    """qkc_set_tile_limit: cap this AC's column tile (0 = default)."""
    _check(lib().qkc_set_tile_limit(ac._h, max_tile_columns))


def set_params(ac: AC, angles, stream=None):
    """angles: float64 CUDA tensor [n_vectors][n_angles] (contiguous)."""
    assert angles.is_cuda and angles.dtype.is_floating_point and angles.is_contiguous()
    n_vec = angles.shape[0] if angles.dim() == 2 else 1
    _check(lib().qkc_set_params(ac._h, _ptr(angles), n_vec, _stream(stream)))
    ac._angles = angles  # keep alive: the gradient reads it


def _cols(col_vec, evidence, ac):
    assert evidence.is_cuda and evidence.is_contiguous() and evidence.shape[-1] == ac.n_vars
    n = evidence.shape[0]
    if col_vec is not None:
        assert col_vec.is_cuda and col_vec.is_contiguous() and col_vec.shape[0] == n
    return n


def evaluate(ac: AC, col_vec, evidence, out=None, stream=None):
    """Upward pass: complex f per column, float64 tensor [n_cols][2]."""
    import torch
    n = _cols(col_vec, evidence, ac)
    if out is None:
        out = torch.empty((n, 2), dtype=torch.float64, device=evidence.device)
    _check(lib().qkc_evaluate(ac._h, _ptr(col_vec), _ptr(evidence), n, _ptr(out), _stream(stream)))
    return out


def reevaluate(ac: AC, angle_slot: int, col_vec, n_cols: int, out=None, stream=None):
    """qkc_reevaluate: after set_params changed one angle slot, recompute only the nodes that depend
    on it, for the columns of the preceding evaluate (same col_vec tensor); float64 [n_cols][2]."""
    import torch
    if out is None:
        out = torch.empty((n_cols, 2), dtype=torch.float64, device=col_vec.device)
    _check(lib().qkc_reevaluate(ac._h, int(angle_slot), _ptr(col_vec), int(n_cols), _ptr(out), _stream(stream)))
    return out


def evaluate_static(ac: AC, col_vec, evidence, out, stream=None):
    """qkc_evaluate_static: the upward pass into the caller's `out` [n_cols][2] float64,
    with the library's fixed device scratch instead of allocated buffers (for callers
    that cannot allocate device memory; see include/qkc.h)."""
    n = _cols(col_vec, evidence, ac)
    _check(lib().qkc_evaluate_static(ac._h, _ptr(col_vec), _ptr(evidence), n, _ptr(out), _stream(stream)))
    return out


def marginals(ac: AC, col_vec, evidence, stream=None):
    """Upward + downward pass: (root [n][2], d f / d lambda [n][n_ind][2])."""
    import torch
    n = _cols(col_vec, evidence, ac)
    root = torch.empty((n, 2), dtype=torch.float64, device=evidence.device)
    marg = torch.empty((n, ac.n_ind, 2), dtype=torch.float64, device=evidence.device)
    _check(lib().qkc_marginals(ac._h, _ptr(col_vec), _ptr(evidence), n, _ptr(root), _ptr(marg), _stream(stream)))
    return root, marg


def gradient(ac: AC, col_vec, evidence, weight, n_vectors: int, stream=None):
    """(value [n_vectors], grad [n_vectors][n_angles]) of sum_c w_c Re f_c per vector."""
    import torch
    n = _cols(col_vec, evidence, ac)
    value = torch.empty((n_vectors,), dtype=torch.float64, device=evidence.device)
    grad = torch.empty((n_vectors, max(1, ac.n_angles)), dtype=torch.float64, device=evidence.device)
    _check(lib().qkc_gradient(ac._h, _ptr(col_vec), _ptr(evidence), _ptr(weight), n, n_vectors, _ptr(value),
                              _ptr(grad), _stream(stream)))
    return value, grad[:, :ac.n_angles]


def sample(ac: AC, seeds, shots, max_shots: int, out=None, stream=None, total_shots: int = 0):
    """Chain-rule samples: uint64 outcome indices [n_vectors][max_shots] (int64 tensor view).
    total_shots: host-known sum of the shots (0: n_vectors x max_shots), sizes the launches."""
    import torch
    n_vec = seeds.shape[0]
    if out is None:
        out = torch.zeros((n_vec, max_shots), dtype=torch.int64, device=seeds.device)
    _check(lib().qkc_sample(ac._h, _ptr(seeds), _ptr(shots), n_vec, max_shots, int(total_shots), _ptr(out),
                            _stream(stream)))
    return out


def sample_probs(ac: AC, seeds, shots, max_shots: int, stream=None, total_shots: int = 0):
    """qkc_sample_probs: (outcome indices [n_vectors][max_shots] int64, each sample's carried
    probability P(x) [n_vectors][max_shots] float64)."""
    import torch
    n_vec = seeds.shape[0]
    out = torch.zeros((n_vec, max_shots), dtype=torch.int64, device=seeds.device)
    probs = torch.zeros((n_vec, max_shots), dtype=torch.float64, device=seeds.device)
    _check(lib().qkc_sample_probs(ac._h, _ptr(seeds), _ptr(shots), n_vec, max_shots, int(total_shots), _ptr(out),
                                  _ptr(probs), _stream(stream)))
    return out, probs


def set_sampler(ac: AC, mode: int, memo_budget_bytes: int = 0):
    """qkc_set_sampler: 1 memoised when estimated cheaper (default), 2 memoised whenever it fits,
    0 one column per prefix group for every node;
    memo_budget_bytes caps the memoised values' device memory (0: automatic)."""
    _check(lib().qkc_set_sampler(ac._h, mode, memo_budget_bytes))


def check_status(ac: AC):
    """qkc_check_status: raise if an earlier sampling call dropped samples (synchronises)."""
    _check(lib().qkc_check_status(ac._h))


def stats_enable(ac: AC, enable: bool = True, max_records: int = 1 << 16):
    """qkc_stats_enable: reset counters; record event-timed level-kernel chains."""
    _check(lib().qkc_stats_enable(ac._h, 1 if enable else 0, max_records))


def get_stats(ac: AC) -> dict:
    """qkc_get_stats: launches, and per pass kind the event time and algorithmic bytes."""
    st = Stats()
    _check(lib().qkc_get_stats(ac._h, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in Stats._fields_}


def gibbs(ac: AC, col_vec, seeds, state, n_sweeps: int, sweep_offset: int = 0, samples=None, stream=None):
    """qkc_gibbs: advance Gibbs chains (one per column) by n_sweeps sweeps; `state` [chains][n_vars]
    int8 is updated in place; returns the outcome index after every sweep [chains][n_sweeps]."""
    import torch
    n = state.shape[0]
    if samples is None:
        samples = torch.zeros((n, n_sweeps), dtype=torch.int64, device=state.device)
    _check(lib().qkc_gibbs(ac._h, _ptr(col_vec), _ptr(seeds), n, _ptr(state), n_sweeps, sweep_offset,
                           _ptr(samples), _stream(stream)))
    return samples
