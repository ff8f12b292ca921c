"""CPU oracle for the ZeroCheck prover (test infrastructure only).

Plain, slow reference implementation of both ZeroCheck forms of the paper
(Fig. side-by-side-zc): the SumCheck prover and verifier (Sec. 3.3, 3.4) and
the NTT prover and verifier (Sec. 3.2).  The arithmetic lives in
``zc_oracle.c``; this module only builds it with gcc and marshals arguments
through ctypes.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and does not import it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "zc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

GATE_PLONK = 1
GATE_PRODUCT = 2
GATE_SUM = 3


def build(force: bool = False) -> str:
    """Compile zc_oracle.c into a shared library (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=gnu11",
                    "-o", tmp, _SRC], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            u32, sz, p = ctypes.c_uint32, ctypes.c_size_t, ctypes.c_void_p
            L.zo_prove_sumcheck.argtypes = [u32, u32, u32, p, p, p, sz, ctypes.POINTER(sz), p, p]
            L.zo_verify_sumcheck.argtypes = [u32, u32, u32, p, p, p, sz, ctypes.POINTER(ctypes.c_int)]
            L.zo_prove_sumcheck_eq.argtypes = [u32, u32, u32, p, p, p, sz, ctypes.POINTER(sz), p, p]
            L.zo_verify_sumcheck_eq.argtypes = [u32, u32, u32, p, p, p, sz, ctypes.POINTER(ctypes.c_int)]
            L.zo_proof_size_eq.argtypes = [u32, u32, u32, ctypes.POINTER(sz)]
            L.zo_pcs_proof_size.argtypes = [u32, u32, u32, u32, ctypes.POINTER(sz)]
            L.zo_pcs_commit.argtypes = [u32, u32, u32, p, p]
            L.zo_pcs_open.argtypes = [u32, u32, u32, u32, p, p, p, p, sz, ctypes.POINTER(sz)]
            L.zo_pcs_verify.argtypes = [u32, u32, u32, u32, p, p, p, p, sz, ctypes.POINTER(ctypes.c_int)]
            L.zo_prove_ntt.argtypes = [u32, u32, u32, u32, p, p, p, sz, ctypes.POINTER(sz), p]
            L.zo_verify_ntt.argtypes = [u32, u32, u32, p, p, p, sz, p, ctypes.POINTER(ctypes.c_int)]
            L.zo_proof_size.argtypes = [u32, u32, u32, u32, ctypes.POINTER(sz)]
            L.zo_fr.argtypes = [ctypes.c_int, p, p, p]
            L.zo_root_of_unity.argtypes = [u32, p]
            L.zo_sha256.argtypes = [p, sz, p]
            L.zo_root.argtypes = [p, sz, p]
            L.zo_ntt.argtypes = [p, u32, ctypes.c_int, p]
            L.zo_coset_lde.argtypes = [p, u32, u32, p]
            L.zo_transcript_demo.argtypes = [u32, u32, u32, u32, u32, p, sz, p]
            _lib = L
    return _lib


def _buf(x) -> np.ndarray:
    a = np.ascontiguousarray(np.frombuffer(x, dtype=np.uint8) if isinstance(x, (bytes, bytearray)) else x)
    return a.view(np.uint8).reshape(-1)


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class _Cols:
    """Keeps the column buffers alive and exposes a ``const uint8_t*[]``."""

    def __init__(self, cols):
        self.arrs = [_buf(c) for c in cols]
        self.ptrs = (ctypes.c_void_p * len(self.arrs))(*[_ptr(a) for a in self.arrs])

    @property
    def p(self):
        return ctypes.cast(self.ptrs, ctypes.c_void_p)


def _roots_buf(roots):
    if roots is None:
        return None, None
    b = np.frombuffer(b"".join(bytes(r) for r in roots), dtype=np.uint8).copy()
    return b, _ptr(b)


def ncols(gate: int, d: int) -> int:
    if gate == GATE_PLONK:
        return 8
    return d + 1 if gate == GATE_PRODUCT else d + (gate >> 8)


def proof_size(form: int, gate: int, n: int, d: int) -> int:
    out = ctypes.c_size_t()
    if lib().zo_proof_size(form, gate, n, d, ctypes.byref(out)) != 0:
        raise ValueError("bad gate/degree")
    return out.value


def prove_sumcheck(gate, n, d, cols, roots=None, with_challenges=False):
    """SumCheck ZeroCheck proof bytes (and r, alpha as canonical bytes)."""
    C = _Cols(cols)
    rb, rp = _roots_buf(roots)
    cap = proof_size(1, gate, n, d)
    proof = np.zeros(cap, np.uint8)
    ln = ctypes.c_size_t()
    r_out = np.zeros(32 * n, np.uint8)
    a_out = np.zeros(32 * n, np.uint8)
    st = lib().zo_prove_sumcheck(gate, n, d, C.p, rp, _ptr(proof), cap, ctypes.byref(ln),
                                 _ptr(r_out), _ptr(a_out))
    if st != 0:
        raise ValueError(f"oracle prove_sumcheck status {st}")
    pb = proof.tobytes()[: ln.value]
    if with_challenges:
        return pb, [r_out[32 * i:32 * i + 32].tobytes() for i in range(n)], \
            [a_out[32 * i:32 * i + 32].tobytes() for i in range(n)]
    return pb


def proof_size_eq(gate: int, n: int, d: int) -> int:
    out = ctypes.c_size_t()
    if lib().zo_proof_size_eq(gate, n, d, ctypes.byref(out)) != 0:
        raise ValueError("bad gate/degree")
    return out.value


def prove_sumcheck_eq(gate, n, d, cols, roots=None, with_challenges=False):
    """Eq-factored SumCheck proof ("ZCS2", transcript v2): rounds carry
    H_i(0..d); optionally also r and alpha as canonical bytes."""
    C = _Cols(cols)
    rb, rp = _roots_buf(roots)
    cap = proof_size_eq(gate, n, d)
    proof = np.zeros(cap, np.uint8)
    ln = ctypes.c_size_t()
    r_out = np.zeros(32 * n, np.uint8)
    a_out = np.zeros(32 * n, np.uint8)
    st = lib().zo_prove_sumcheck_eq(gate, n, d, C.p, rp, _ptr(proof), cap, ctypes.byref(ln),
                                    _ptr(r_out), _ptr(a_out))
    if st != 0:
        raise ValueError(f"oracle prove_sumcheck_eq status {st}")
    pb = proof.tobytes()[: ln.value]
    if with_challenges:
        return pb, [r_out[32 * i:32 * i + 32].tobytes() for i in range(n)], \
            [a_out[32 * i:32 * i + 32].tobytes() for i in range(n)]
    return pb


def verify_sumcheck_eq(gate, n, d, cols, proof, roots=None) -> bool:
    C = _Cols(cols)
    rb, rp = _roots_buf(roots)
    pr = _buf(proof)
    acc = ctypes.c_int(0)
    st = lib().zo_verify_sumcheck_eq(gate, n, d, C.p, rp, _ptr(pr), pr.size, ctypes.byref(acc))
    if st != 0:
        return False
    return bool(acc.value)


# ---- hash-based PCS around the ZeroCheck (Ligero-style; see zc_oracle.c)

def pcs_default_nc(n: int) -> int:
    return min(n, 12)


def pcs_proof_size(n: int, c: int, t: int, nc: int | None = None) -> int:
    out = ctypes.c_size_t()
    if lib().zo_pcs_proof_size(n, nc or pcs_default_nc(n), c, t, ctypes.byref(out)) != 0:
        raise ValueError("bad PCS shape")
    return out.value


def pcs_commit(n: int, cols, nc: int | None = None) -> bytes:
    """Merkle root over the rate-1/4 row encodings of the c columns."""
    C = _Cols(cols)
    root = np.zeros(32, np.uint8)
    if lib().zo_pcs_commit(n, nc or pcs_default_nc(n), len(cols), C.p, _ptr(root)) != 0:
        raise ValueError("pcs_commit rejected its input")
    return root.tobytes()


def pcs_open(n: int, cols, alpha, values, t: int, nc: int | None = None) -> bytes:
    """Opening of every column at alpha (canonical bytes, n of them) with the
    claimed values (canonical bytes, one per column), t queried columns."""
    C = _Cols(cols)
    a = np.frombuffer(b"".join(bytes(x) for x in alpha), dtype=np.uint8).copy()
    v = np.frombuffer(b"".join(bytes(x) for x in values), dtype=np.uint8).copy()
    cap = pcs_proof_size(n, len(cols), t, nc)
    out = np.zeros(cap, np.uint8)
    ln = ctypes.c_size_t()
    st = lib().zo_pcs_open(n, nc or pcs_default_nc(n), len(cols), t, C.p, _ptr(a), _ptr(v), _ptr(out), cap,
                           ctypes.byref(ln))
    if st != 0:
        raise ValueError(f"oracle pcs_open status {st}")
    return out.tobytes()[: ln.value]


def pcs_verify(n: int, c: int, t: int, root: bytes, alpha, values, proof, nc: int | None = None) -> bool:
    a = np.frombuffer(b"".join(bytes(x) for x in alpha), dtype=np.uint8).copy()
    v = np.frombuffer(b"".join(bytes(x) for x in values), dtype=np.uint8).copy()
    r = np.frombuffer(bytes(root), dtype=np.uint8).copy()
    pr = _buf(proof)
    acc = ctypes.c_int(0)
    st = lib().zo_pcs_verify(n, nc or pcs_default_nc(n), c, t, _ptr(r), _ptr(a), _ptr(v), _ptr(pr), pr.size,
                             ctypes.byref(acc))
    return st == 0 and bool(acc.value)


def verify_sumcheck(gate, n, d, cols, proof, roots=None) -> bool:
    C = _Cols(cols)
    rb, rp = _roots_buf(roots)
    pr = _buf(proof)
    acc = ctypes.c_int(0)
    st = lib().zo_verify_sumcheck(gate, n, d, C.p, rp, _ptr(pr), pr.size, ctypes.byref(acc))
    if st != 0:
        return False
    return bool(acc.value)


def domain_word(k: int, s: int | None = None) -> int:
    """Domain word of the NTT form: 2^k N points, or with s (< k) the
    step-radix domain of 2^k N + 2^s N points."""
    return k if s is None else k | ((s + 1) << 8)


def domain_size(n: int, d: int, log_blowup: int = 0) -> int:
    """Number of points M of the NTT domain for a domain word (0: default)."""
    k, sp1 = log_blowup & 0xFF, (log_blowup >> 8) & 0xFF
    if not sp1:
        return 1 << (n + (k or (max(d, 1) - 1).bit_length()))
    return (1 << (n + k)) + (1 << (n + sp1 - 1))


def prove_ntt(gate, n, d, cols, roots=None, log_blowup=0):
    """NTT ZeroCheck proof bytes and the quotient q (canonical, M*32 bytes).
    log_blowup is the domain word (see domain_word); 0 selects the default."""
    C = _Cols(cols)
    rb, rp = _roots_buf(roots)
    M = domain_size(n, d, log_blowup)
    cap = proof_size(2, gate, n, d)
    proof = np.zeros(cap, np.uint8)
    q = np.zeros(M * 32, np.uint8)
    ln = ctypes.c_size_t()
    st = lib().zo_prove_ntt(gate, n, d, log_blowup, C.p, rp, _ptr(proof), cap, ctypes.byref(ln), _ptr(q))
    if st != 0:
        raise ValueError(f"oracle prove_ntt status {st}")
    return proof.tobytes()[: ln.value], q


def verify_ntt(gate, n, d, cols, proof, q, roots=None) -> bool:
    C = _Cols(cols)
    rb, rp = _roots_buf(roots)
    pr = _buf(proof)
    qb = _buf(q)
    acc = ctypes.c_int(0)
    st = lib().zo_verify_ntt(gate, n, d, C.p, rp, _ptr(pr), pr.size, _ptr(qb), ctypes.byref(acc))
    if st != 0:
        return False
    return bool(acc.value)


# ---- hooks used by the pin tests (canonical integers in and out) ----

def _to32(x: int) -> np.ndarray:
    return np.frombuffer(int(x).to_bytes(32, "little"), dtype=np.uint8).copy()


def _from32(a) -> int:
    return int.from_bytes(bytes(a), "little")


def fr(op: str, a: int, b: int | None = None) -> int:
    code = {"add": 0, "sub": 1, "mul": 2, "inv": 3, "neg": 4}[op]
    A = _to32(a)
    B = _to32(b) if b is not None else None
    out = np.zeros(32, np.uint8)
    st = lib().zo_fr(code, _ptr(A), _ptr(B) if B is not None else None, _ptr(out))
    if st != 0:
        raise ValueError("oracle field op rejected input")
    return _from32(out)


def root_of_unity(logn: int) -> int:
    out = np.zeros(32, np.uint8)
    if lib().zo_root_of_unity(logn, _ptr(out)) != 0:
        raise ValueError
    return _from32(out)


def sha256(msg: bytes) -> bytes:
    m = np.frombuffer(bytes(msg) or b"\0", dtype=np.uint8).copy()
    out = np.zeros(32, np.uint8)
    lib().zo_sha256(_ptr(m), len(msg), _ptr(out))
    return out.tobytes()


def root(v) -> bytes:
    a = _buf(v)
    out = np.zeros(32, np.uint8)
    if lib().zo_root(_ptr(a), a.size // 32, _ptr(out)) != 0:
        raise ValueError("root needs a non-empty vector")
    return out.tobytes()


def ints_to_bytes(xs) -> np.ndarray:
    return np.frombuffer(b"".join(int(x).to_bytes(32, "little") for x in xs), dtype=np.uint8).copy()


def bytes_to_ints(b) -> list[int]:
    b = bytes(_buf(b))
    return [int.from_bytes(b[i:i + 32], "little") for i in range(0, len(b), 32)]


def ntt(values, logn: int, inverse: bool = False) -> list[int]:
    a = ints_to_bytes(values)
    out = np.zeros_like(a)
    if lib().zo_ntt(_ptr(a), logn, 1 if inverse else 0, _ptr(out)) != 0:
        raise ValueError
    return bytes_to_ints(out)


def coset_lde(coeffs, n: int, logm: int) -> list[int]:
    a = ints_to_bytes(coeffs)
    out = np.zeros(32 << logm, np.uint8)
    if lib().zo_coset_lde(_ptr(a), n, logm, _ptr(out)) != 0:
        raise ValueError
    return bytes_to_ints(out)


def transcript_demo(form, gate, n, d, logm, msg: bytes) -> int:
    m = np.frombuffer(bytes(msg) or b"\0", dtype=np.uint8).copy()
    out = np.zeros(32, np.uint8)
    lib().zo_transcript_demo(form, gate, n, d, logm, _ptr(m), len(msg), _ptr(out))
    return _from32(out)


def num_threads() -> int:
    return int(lib().zo_num_threads())
