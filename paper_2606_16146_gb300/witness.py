"""Seeded synthetic ZeroCheck witnesses (input generator).

Shared by the tests, the benchmark and the oracle runs; holds no prover
arithmetic.  The C source ``csrc/witness.c`` documents the distribution:
uniform field elements from per-column splitmix64 streams, with the last
column solved so that the gate vanishes on the whole domain (Plonk:
c = -(qL a + qR b + qM a b + qC)/qO; product gate: o = q w1 ... w_{d-1};
sum gate: the last single column is minus the rest, or with no single
column one factor is zeroed at every point).
Columns come back as ``numpy.uint8`` arrays of N*32 canonical little-endian
bytes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "witness.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libzcwitness.so")
_lock = threading.Lock()
_lib = None

GATE_PLONK = 1
GATE_PRODUCT = 2
GATE_SUM = 3


def gate_sum(m: int) -> int:
    """Gate word of the sum gate g_1 ... g_d + g_{d+1} + ... + g_{d+m}."""
    return GATE_SUM | (m << 8)


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=gnu11", "-o", tmp, _SRC],
                   check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            L.zw_generate.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]
            L.zw_generate_edge.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                           ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]
            _lib = L
    return _lib


def ncols(gate: int, d: int) -> int:
    if gate == GATE_PLONK:
        return 8
    return d + 1 if gate == GATE_PRODUCT else d + (gate >> 8)


def generate(gate: int, n: int, d: int, seed: int, tamper: bool = False) -> list[np.ndarray]:
    """Return the c columns of a satisfying (or, with ``tamper``, a violating) witness."""
    c = ncols(gate, d)
    N = 1 << n
    cols = [np.empty(N * 32, dtype=np.uint8) for _ in range(c)]
    ptrs = (ctypes.c_void_p * c)(*[a.ctypes.data for a in cols])
    st = _load().zw_generate(gate, n, d, seed & (2**64 - 1), 1 if tamper else 0,
                             ctypes.cast(ptrs, ctypes.c_void_p))
    if st != 0:
        raise ValueError(f"witness generation failed (status {st})")
    return cols


def generate_edge(gate: int, n: int, d: int, seed: int, only_edges: bool = False) -> list[np.ndarray]:
    """Columns of boundary field values (0, 1, r-1, r-2^k, 2^k, 2^256 mod r, ...),
    half of the elements uniform unless ``only_edges``; the gate does not vanish."""
    c = ncols(gate, d)
    N = 1 << n
    cols = [np.empty(N * 32, dtype=np.uint8) for _ in range(c)]
    ptrs = (ctypes.c_void_p * c)(*[a.ctypes.data for a in cols])
    st = _load().zw_generate_edge(gate, n, d, seed & (2**64 - 1), 1 if only_edges else 0,
                                  ctypes.cast(ptrs, ctypes.c_void_p))
    if st != 0:
        raise ValueError(f"edge witness generation failed (status {st})")
    return cols


def default_seed(gate: int, n: int, d: int) -> int:
    """Seeds of the standard workloads: Plonk 1000+n, product gate 2000+d."""
    return 1000 + n if gate == GATE_PLONK else 2000 + d
