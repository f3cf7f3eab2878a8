"""ctypes binding of acref.c, the plain FP64 AC evaluator (oracle; test
infrastructure only).  Built in-tree with gcc into oracle/_build/."""
from __future__ import annotations

import ctypes
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "acref.c"
BUILD = HERE / "_build"
LIB = BUILD / "libacref.so"
_lib = None


def build(force: bool = False) -> Path:
    BUILD.mkdir(exist_ok=True)
    if force or not LIB.exists() or LIB.stat().st_mtime < SRC.stat().st_mtime:
        tmp = BUILD / "libacref.so.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", str(SRC), "-o", str(tmp), "-lm"],
                       check=True, capture_output=True)
        tmp.replace(LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(LIB))
        P = ctypes.c_void_p
        L.oac_open.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(P)]
        L.oac_open.restype = ctypes.c_int
        L.oac_close.argtypes = [P]
        L.oac_close.restype = None
        L.oac_info.argtypes = [P, P]
        L.oac_info.restype = None
        L.oac_up.argtypes = [P, P, P, P]
        L.oac_up.restype = None
        L.oac_values.argtypes = [P, P]
        L.oac_values.restype = None
        L.oac_marginals.argtypes = [P, P, P, P, P]
        L.oac_marginals.restype = None
        L.oac_gradient.argtypes = [P, P, P, ctypes.c_double, P, P]
        L.oac_gradient.restype = None
        L.oac_sample.argtypes = [P, P, ctypes.c_uint64, ctypes.c_int32, P]
        L.oac_sample.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class ACRef:
    """One compiled AC, evaluated one column at a time in FP64."""

    def __init__(self, ac_bytes: bytes):
        self._buf = ctypes.create_string_buffer(ac_bytes, len(ac_bytes))
        self._h = ctypes.c_void_p()
        st = lib().oac_open(self._buf, len(ac_bytes), ctypes.byref(self._h))
        if st != 0:
            raise ValueError(f"oac_open failed ({st})")
        info = np.zeros(10, dtype=np.int64)
        lib().oac_info(self._h, _p(info))
        (self.kind, self.n_qubits, self.n_angles, self.n_vars, self.n_ind, self.n_nodes, self.n_edges,
         self.n_levels, self.n_leaves, self.root) = map(int, info)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().oac_close(self._h)
            self._h = None

    def _ang(self, angles):
        a = np.ascontiguousarray(np.asarray(angles, dtype=np.float64).reshape(-1))
        if a.size == 0:
            a = np.zeros(1)
        return a

    def _ev(self, evidence):
        e = np.ascontiguousarray(np.asarray(evidence, dtype=np.int8).reshape(-1))
        assert e.size == self.n_vars
        return e

    def up(self, angles, evidence) -> complex:
        out = np.zeros(2)
        lib().oac_up(self._h, _p(self._ang(angles)), _p(self._ev(evidence)), _p(out))
        return complex(out[0], out[1])

    def values(self) -> np.ndarray:
        out = np.zeros((self.n_nodes, 2))
        lib().oac_values(self._h, _p(out))
        return out[:, 0] + 1j * out[:, 1]

    def marginals(self, angles, evidence):
        root = np.zeros(2)
        adj = np.zeros((self.n_ind, 2))
        lib().oac_marginals(self._h, _p(self._ang(angles)), _p(self._ev(evidence)), _p(root), _p(adj))
        return complex(root[0], root[1]), adj[:, 0] + 1j * adj[:, 1]

    def gradient(self, angles, evidence, weight=1.0):
        value = np.zeros(1)
        grad = np.zeros(max(1, self.n_angles))
        lib().oac_gradient(self._h, _p(self._ang(angles)), _p(self._ev(evidence)), float(weight), _p(value),
                           _p(grad))
        return float(value[0]), grad[:self.n_angles]

    def sample(self, angles, seed: int, shots: int) -> np.ndarray:
        bits = np.zeros(max(1, shots), dtype=np.uint64)
        st = lib().oac_sample(self._h, _p(self._ang(angles)), ctypes.c_uint64(int(seed)), shots, _p(bits))
        if st != 0:
            raise MemoryError("oac_sample")
        return bits[:shots]


# ---------------------------------------------------------------- many columns on the host cores
_worker_ac = {}


def _worker(job):
    """One job of a spawned pool: ("sample", angles, seed, shots) or ("up", angles, evidence)."""
    key, ac_bytes, task = job
    if key not in _worker_ac:
        _worker_ac.clear()
        _worker_ac[key] = ACRef(ac_bytes)
    ref = _worker_ac[key]
    if task[0] == "sample":
        return ref.sample(task[1], task[2], task[3])
    return ref.up(task[1], task[2])


def run_many(ac_bytes: bytes, tasks, processes: int = 0):
    """Run oracle tasks -- ("sample", angles, seed, shots) or ("up", angles, evidence) -- on one
    spawn-started process per host core (a process forked from one holding a CUDA context can
    hang; spawn starts clean ones).  Results in task order.  The evaluator itself is unchanged:
    each task is one plain call of ACRef.sample or ACRef.up."""
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    procs = processes or min(len(tasks), os.cpu_count() or 1)
    key = hash(ac_bytes)
    jobs = [(key, ac_bytes, t) for t in tasks]
    if procs <= 1:
        return [_worker(j) for j in jobs]
    # an executor (unlike multiprocessing.Pool) raises when a worker dies instead of waiting forever
    with ProcessPoolExecutor(procs, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_worker, jobs, chunksize=1))
