"""Python binding of libzc.so (the C ABI declared in include/zc.h).

Argument marshalling only: every step of proving runs in the library's CUDA
kernels.  Columns may be ``torch.Tensor`` objects on a CUDA device (passed by
``data_ptr()``) or host buffers (``numpy`` arrays, ``bytes``); the proof
buffer is host memory unless a device tensor is given.  There is no CPU
fallback: importing this module on a machine without the built library
raises, and every call reports the library's status code as an exception.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

ZC_OK = 0
STATUS = {0: "ZC_OK", 1: "ZC_ERR_ARG", 2: "ZC_ERR_OOM", 3: "ZC_ERR_CUDA", 4: "ZC_ERR_TIMEOUT",
          5: "ZC_ERR_UNSUPPORTED", 6: "ZC_ERR_BUFFER_TOO_SMALL"}
(ZC_ERR_ARG, ZC_ERR_OOM, ZC_ERR_CUDA, ZC_ERR_TIMEOUT, ZC_ERR_UNSUPPORTED,
 ZC_ERR_BUFFER_TOO_SMALL) = 1, 2, 3, 4, 5, 6
ZC_GATE_PLONK, ZC_GATE_PRODUCT, ZC_GATE_SUM = 1, 2, 3


def gate_sum(m: int) -> int:
    """ZC_GATE_SUM_OF(m): gate word of g_1 ... g_d + g_{d+1} + ... + g_{d+m}."""
    return ZC_GATE_SUM | (m << 8)


ZC_FORM_SUMCHECK, ZC_FORM_NTT, ZC_FORM_SUMCHECK_EQ = 1, 2, 3
ZC_TUNE_SC_GRID, ZC_TUNE_SC_TAIL_LOG, ZC_TUNE_NTT_TILE_LOG, ZC_TUNE_NTT_MINB = 1, 2, 3, 4
ZC_TUNE_SC_SMALL_LOG, ZC_TUNE_SC_MINB, ZC_TUNE_SC_PROD_PPT, ZC_TUNE_SC_CHUNK_LOG = 5, 6, 7, 8
ZC_TUNE_BATCH_LANES, ZC_TUNE_SC_QUAD_LOG, ZC_TUNE_SC_PROD_FUSE, ZC_TUNE_NTT_TWO_LOG = 9, 10, 11, 12


class ZCError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class zc_params(ctypes.Structure):
    _fields_ = [("gate", ctypes.c_uint32), ("n", ctypes.c_uint32), ("d", ctypes.c_uint32),
                ("log_blowup", ctypes.c_uint32)]


class zc_setup_opts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("max_n", ctypes.c_uint32), ("max_d", ctypes.c_uint32),
                ("mem_budget_bytes", ctypes.c_uint64)]


class zc_request(ctypes.Structure):
    _fields_ = [("arrival_s", ctypes.c_double), ("params", zc_params), ("form", ctypes.c_int),
                ("cols", ctypes.c_void_p), ("proof", ctypes.c_void_p), ("q_out", ctypes.c_void_p)]


class zc_result(ctypes.Structure):
    _fields_ = [("admit_s", ctypes.c_double), ("done_s", ctypes.c_double),
                ("scratch_bytes", ctypes.c_uint64), ("slot", ctypes.c_uint32),
                ("waited_for_memory", ctypes.c_uint32), ("status", ctypes.c_int)]


class zc_pcs_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("nc", ctypes.c_uint32), ("c", ctypes.c_uint32), ("t", ctypes.c_uint32)]


class zc_serve_opts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_uint32), ("hbm_budget_bytes", ctypes.c_uint64),
                ("in_order", ctypes.c_uint32), ("timeout_s", ctypes.c_double),
                ("priority_bytes", ctypes.c_uint64)]


_lib = None


def lib(path: str | None = None):
    """Load libzc.so (building it first if it is missing)."""
    global _lib
    if _lib is None:
        p = path or _build.LIB
        if not os.path.exists(p):
            _build.build()
        L = ctypes.CDLL(p)
        vp, sz, u8p = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p
        P = ctypes.POINTER
        L.zc_setup.argtypes = [P(zc_setup_opts), P(vp)]
        L.zc_setup.restype = ctypes.c_int
        L.zc_destroy.argtypes = [vp]
        L.zc_destroy.restype = None
        L.zc_proof_size.argtypes = [P(zc_params), ctypes.c_int, P(sz)]
        L.zc_proof_size.restype = ctypes.c_int
        L.zc_prove_sumcheck.argtypes = [vp, P(zc_params), vp, ctypes.c_int, vp, vp, u8p, sz, P(sz)]
        L.zc_prove_sumcheck.restype = ctypes.c_int
        L.zc_prove_sumcheck_eq.argtypes = [vp, P(zc_params), vp, ctypes.c_int, vp, vp, u8p, sz, P(sz)]
        L.zc_prove_sumcheck_eq.restype = ctypes.c_int
        L.zc_prove_ntt.argtypes = [vp, P(zc_params), vp, ctypes.c_int, vp, vp, u8p, sz, P(sz), vp,
                                   ctypes.c_int]
        L.zc_prove_ntt.restype = ctypes.c_int
        L.zc_verify.argtypes = [P(zc_params), ctypes.c_int, vp, vp, u8p, sz, vp, P(ctypes.c_int)]
        L.zc_verify.restype = ctypes.c_int
        L.zc_roots.argtypes = [vp, P(zc_params), vp, ctypes.c_int, vp, vp]
        L.zc_roots.restype = ctypes.c_int
        L.zc_scratch_bytes.argtypes = [vp, P(zc_params), ctypes.c_int, ctypes.c_int, P(sz)]
        L.zc_scratch_bytes.restype = ctypes.c_int
        L.zc_serve.argtypes = [vp, P(zc_request), ctypes.c_uint32, P(zc_serve_opts), P(zc_result)]
        L.zc_serve.restype = ctypes.c_int
        L.zc_tune_set.argtypes = [vp, ctypes.c_int, ctypes.c_uint32, ctypes.c_int, ctypes.c_int32]
        L.zc_tune_set.restype = ctypes.c_int
        L.zc_tune_get.argtypes = [vp, ctypes.c_int, ctypes.c_uint32, ctypes.c_int, P(ctypes.c_int32)]
        L.zc_tune_get.restype = ctypes.c_int
        L.zc_stats.argtypes = [vp, P(ctypes.c_double), ctypes.c_uint32]
        L.zc_stats.restype = ctypes.c_int
        L.zc_prove_batch.argtypes = [vp, ctypes.c_uint32, vp, vp, vp, vp, vp, vp]
        L.zc_prove_batch.restype = ctypes.c_int
        L.zc_batch_create.argtypes = [vp, ctypes.c_uint32, vp, vp, vp, vp, vp, P(vp)]
        L.zc_batch_create.restype = ctypes.c_int
        L.zc_batch_launch.argtypes = [vp, vp]
        L.zc_batch_launch.restype = ctypes.c_int
        L.zc_batch_kernels.argtypes = [vp]
        L.zc_batch_kernels.restype = ctypes.c_uint32
        L.zc_batch_destroy.argtypes = [vp]
        L.zc_batch_destroy.restype = None
        L.zc_prove_sumcheck_static.argtypes = [P(zc_params), vp, vp, vp, u8p, sz, P(sz)]
        L.zc_prove_sumcheck_static.restype = ctypes.c_int
        L.zc_pcs_proof_size.argtypes = [P(zc_pcs_params), P(sz)]
        L.zc_pcs_proof_size.restype = ctypes.c_int
        L.zc_pcs_commit.argtypes = [vp, P(zc_pcs_params), vp, ctypes.c_int, vp, P(vp), u8p]
        L.zc_pcs_commit.restype = ctypes.c_int
        L.zc_pcs_open.argtypes = [vp, vp, vp, vp, u8p, sz, P(sz)]
        L.zc_pcs_open.restype = ctypes.c_int
        L.zc_pcs_verify.argtypes = [P(zc_pcs_params), u8p, vp, vp, u8p, sz, P(ctypes.c_int)]
        L.zc_pcs_verify.restype = ctypes.c_int
        L.zc_pcs_destroy.argtypes = [vp]
        L.zc_pcs_destroy.restype = None
        L.zc_sumcheck_point.argtypes = [P(zc_params), ctypes.c_int, vp, u8p, sz, vp, vp, P(ctypes.c_int)]
        L.zc_sumcheck_point.restype = ctypes.c_int
        L.zc_last_error.argtypes = [vp]
        L.zc_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _addr(x) -> int:
    if _is_torch(x):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"unsupported buffer type {type(x)}")


def _host_array(x) -> np.ndarray:
    if isinstance(x, (bytes, bytearray)):
        return np.frombuffer(bytes(x), dtype=np.uint8)
    return np.ascontiguousarray(x)


class _Ptrs:
    def __init__(self, bufs):
        self.keep = list(bufs)
        self.arr = (ctypes.c_void_p * len(self.keep))(*[_addr(b) for b in self.keep])

    @property
    def p(self):
        return ctypes.cast(self.arr, ctypes.c_void_p)


def _roots_arg(roots):
    if roots is None:
        return None, None
    b = np.frombuffer(b"".join(bytes(r) for r in roots), dtype=np.uint8).copy()
    return b, b.ctypes.data


def _stream_ptr(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


def domain_word(k: int, s: int | None = None) -> int:
    """zc_params.log_blowup for 2^k N points, or with s (< k) the step-radix
    domain of 2^k N + 2^s N points (ZC_DOMAIN_STEP(k, s))."""
    return k if s is None else k | ((s + 1) << 8)


def domain_size(n: int, d: int, log_blowup: int = 0) -> int:
    """Points M of the NTT domain (the quotient has M coefficients)."""
    k, sp1 = log_blowup & 0xFF, (log_blowup >> 8) & 0xFF
    if not sp1:
        return 1 << (n + (k or (d - 1).bit_length()))
    return (1 << (n + k)) + (1 << (n + sp1 - 1))


def proof_size(gate, n, d, form, log_blowup=0) -> int:
    p = zc_params(gate, n, d, log_blowup)
    out = ctypes.c_size_t()
    st = lib().zc_proof_size(ctypes.byref(p), form, ctypes.byref(out))
    if st != ZC_OK:
        raise ZCError(st, "zc_proof_size")
    return out.value


class Context:
    """A zc_ctx: owns device scratch, constants and events for one GPU."""

    def __init__(self, device: int = 0, max_n: int = 24, max_d: int = 8, mem_budget_bytes: int = 0):
        opts = zc_setup_opts(device, max_n, max_d, mem_budget_bytes)
        h = ctypes.c_void_p()
        st = lib().zc_setup(ctypes.byref(opts), ctypes.byref(h))
        if st != ZC_OK:
            raise ZCError(st, "zc_setup")
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            lib().zc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != ZC_OK:
            msg = lib().zc_last_error(self.h)
            raise ZCError(st, f"{what}: {msg.decode() if msg else ''}")

    def _cols(self, cols):
        on_dev = all(_is_torch(c) and c.is_cuda for c in cols)
        if not on_dev:
            cols = [_host_array(c) for c in cols]
        return _Ptrs(cols), 1 if on_dev else 0

    def prove_sumcheck(self, gate, n, d, cols, roots=None, stream=None, proof_out=None, eq_factored=False):
        """SumCheck-form proof.  Returns the proof (numpy uint8) unless proof_out
        (a device tensor) is given, in which case the call is asynchronous.
        eq_factored: zc_prove_sumcheck_eq (rounds carry H_i(0..d), "ZCS2")."""
        p = zc_params(gate, n, d, 0)
        P, on_dev = self._cols(cols)
        rb, rp = _roots_arg(roots)
        form = ZC_FORM_SUMCHECK_EQ if eq_factored else ZC_FORM_SUMCHECK
        cap = proof_size(gate, n, d, form)
        out = proof_out if proof_out is not None else np.zeros(cap, np.uint8)
        ln = ctypes.c_size_t()
        fn = lib().zc_prove_sumcheck_eq if eq_factored else lib().zc_prove_sumcheck
        st = fn(self.h, ctypes.byref(p), P.p, on_dev, rp, _stream_ptr(stream), _addr(out), cap, ctypes.byref(ln))
        self._check(st, "zc_prove_sumcheck_eq" if eq_factored else "zc_prove_sumcheck")
        return out

    def prove_ntt(self, gate, n, d, cols, roots=None, stream=None, proof_out=None, q_out=None,
                  log_blowup=0, want_q=True):
        """NTT-form proof.  Returns (proof, q); q_out may be a device tensor of
        M*32 bytes, or None for a host array; want_q=False keeps q on the
        device only (returns (proof, None))."""
        p = zc_params(gate, n, d, log_blowup)
        P, on_dev = self._cols(cols)
        rb, rp = _roots_arg(roots)
        cap = proof_size(gate, n, d, ZC_FORM_NTT, log_blowup)
        M = domain_size(n, d, log_blowup)
        out = proof_out if proof_out is not None else np.zeros(cap, np.uint8)
        q = q_out if q_out is not None else (np.zeros(M * 32, np.uint8) if want_q else None)
        q_dev = 1 if (q is None or (_is_torch(q) and q.is_cuda)) else 0
        ln = ctypes.c_size_t()
        st = lib().zc_prove_ntt(self.h, ctypes.byref(p), P.p, on_dev, rp, _stream_ptr(stream),
                                _addr(out), cap, ctypes.byref(ln), _addr(q) if q is not None else None,
                                q_dev)
        self._check(st, "zc_prove_ntt")
        return out, q

    def pcs_commit(self, n, cols, t, nc=0, stream=None) -> "PcsCommitment":
        """Commit to the columns with the hash-based PCS (zc_pcs_commit)."""
        return PcsCommitment(self, n, cols, t, nc, stream)

    def roots(self, gate, n, d, cols, stream=None) -> list[bytes]:
        p = zc_params(gate, n, d, 0)
        P, on_dev = self._cols(cols)
        c = len(cols)
        out = np.zeros(32 * c, np.uint8)
        st = lib().zc_roots(self.h, ctypes.byref(p), P.p, on_dev, _stream_ptr(stream), out.ctypes.data)
        self._check(st, "zc_roots")
        return [out[32 * j:32 * j + 32].tobytes() for j in range(c)]

    def _batch_args(self, forms, params, cols, proofs, q_outs):
        n = len(forms)
        F = (ctypes.c_int * n)(*forms)
        Pa = (zc_params * n)(*[zc_params(g, nn, d, lb) for (g, nn, d, lb) in params])
        inner = [_Ptrs(c) for c in cols]
        C = (ctypes.c_void_p * n)(*[ctypes.cast(x.arr, ctypes.c_void_p).value for x in inner])
        Pr = (ctypes.c_void_p * n)(*[_addr(p) for p in proofs])
        Q = None
        if q_outs is not None:
            Q = (ctypes.c_void_p * n)(*[(_addr(q) if q is not None else None) for q in q_outs])
        keep = (F, Pa, inner, C, Pr, Q)
        return keep, F, Pa, C, Pr, Q

    def prove_batch(self, forms, params, cols, proofs, q_outs=None, stream=None):
        """Prove a batch (device columns, proofs and q).  params: (gate, n, d, log_blowup)."""
        keep, F, Pa, C, Pr, Q = self._batch_args(forms, params, cols, proofs, q_outs)
        st = lib().zc_prove_batch(self.h, len(forms), ctypes.cast(F, ctypes.c_void_p),
                                  ctypes.cast(Pa, ctypes.c_void_p), ctypes.cast(C, ctypes.c_void_p),
                                  _stream_ptr(stream), ctypes.cast(Pr, ctypes.c_void_p),
                                  ctypes.cast(Q, ctypes.c_void_p) if Q is not None else None)
        self._check(st, "zc_prove_batch")

    def batch_graph(self, forms, params, cols, proofs, q_outs=None):
        """Capture the batch into one CUDA graph; returns a BatchGraph."""
        keep, F, Pa, C, Pr, Q = self._batch_args(forms, params, cols, proofs, q_outs)
        h = ctypes.c_void_p()
        st = lib().zc_batch_create(self.h, len(forms), ctypes.cast(F, ctypes.c_void_p),
                                   ctypes.cast(Pa, ctypes.c_void_p), ctypes.cast(C, ctypes.c_void_p),
                                   ctypes.cast(Pr, ctypes.c_void_p),
                                   ctypes.cast(Q, ctypes.c_void_p) if Q is not None else None,
                                   ctypes.byref(h))
        self._check(st, "zc_batch_create")
        return BatchGraph(h, keep)

    def scratch_bytes(self, gate, n, d, form, q_on_device=False, log_blowup=0) -> int:
        """Device scratch one proof of this shape takes (its admission footprint)."""
        out = ctypes.c_size_t()
        p = zc_params(gate, n, d, log_blowup)
        self._check(lib().zc_scratch_bytes(self.h, ctypes.byref(p), form, 1 if q_on_device else 0,
                                           ctypes.byref(out)), "zc_scratch_bytes")
        return int(out.value)

    def serve(self, requests, slots=8, hbm_budget_bytes=180 << 30, in_order=False, timeout_s=0.0,
              priority_bytes=0):
        """Run the request loop.  requests: dicts with arrival_s, gate, n, d, form, cols
        (device tensors), proof (device tensor) and optional q (device tensor).  Returns one
        dict per request: admit_s, done_s, scratch_bytes, slot, waited_for_memory, status.
        priority_bytes > 0: requests with at least that much scratch run one at a time on
        the high-priority slot 0, the others on slots 1.."""
        cnt = len(requests)
        R = (zc_request * max(1, cnt))()
        keep = []
        for i, r in enumerate(requests):
            cp = _Ptrs(r["cols"])
            keep.append(cp)
            R[i].arrival_s = float(r["arrival_s"])
            R[i].params = zc_params(r["gate"], r["n"], r["d"], r.get("log_blowup", 0))
            R[i].form = int(r["form"])
            R[i].cols = ctypes.cast(cp.arr, ctypes.c_void_p).value
            R[i].proof = _addr(r["proof"])
            R[i].q_out = _addr(r["q"]) if r.get("q") is not None else None
        out = (zc_result * max(1, cnt))()
        o = zc_serve_opts(slots, hbm_budget_bytes, 1 if in_order else 0, timeout_s, priority_bytes)
        st = lib().zc_serve(self.h, R, cnt, ctypes.byref(o), out)
        res = [{"admit_s": out[i].admit_s, "done_s": out[i].done_s,
                "scratch_bytes": int(out[i].scratch_bytes), "slot": int(out[i].slot),
                "waited_for_memory": bool(out[i].waited_for_memory), "status": int(out[i].status)}
               for i in range(cnt)]
        if st != ZC_OK:
            msg = lib().zc_last_error(self.h)
            err = ZCError(st, f"zc_serve: {msg.decode() if msg else ''}")
            err.results = res
            raise err
        return res

    def tune_set(self, form: int, n: int, key: int, value: int) -> None:
        """Launch parameter for proofs of (form, n); n = 0 for every size, value 0 clears."""
        self._check(lib().zc_tune_set(self.h, form, n, key, value), "zc_tune_set")

    def tune_get(self, form: int, n: int, key: int) -> int:
        v = ctypes.c_int32()
        self._check(lib().zc_tune_get(self.h, form, n, key, ctypes.byref(v)), "zc_tune_get")
        return int(v.value)

    def stats(self) -> list[float]:
        a = (ctypes.c_double * 10)()
        self._check(lib().zc_stats(self.h, a, 10), "zc_stats")
        return list(a)


class BatchGraph:
    """A batch captured as one CUDA graph (zc_batch)."""

    def __init__(self, h, keep):
        self.h = h
        self._keep = keep

    def launch(self, stream=None):
        st = lib().zc_batch_launch(self.h, _stream_ptr(stream))
        if st != ZC_OK:
            raise ZCError(st, "zc_batch_launch")

    @property
    def kernels(self) -> int:
        return int(lib().zc_batch_kernels(self.h))

    def close(self):
        if self.h:
            lib().zc_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def verify(gate, n, d, form, cols, proof, q=None, roots=None, log_blowup=0) -> bool:
    """Host-side verifier (no GPU needed).  cols/q: host buffers."""
    p = zc_params(gate, n, d, log_blowup)
    P = _Ptrs([_host_array(c) for c in cols])
    rb, rp = _roots_arg(roots)
    pr = _host_array(proof)
    qa = _host_array(q) if q is not None else None
    acc = ctypes.c_int(0)
    st = lib().zc_verify(ctypes.byref(p), form, P.p, rp, pr.ctypes.data, pr.size,
                         qa.ctypes.data if qa is not None else None, ctypes.byref(acc))
    if st == 1:
        return False
    if st != ZC_OK:
        raise ZCError(st, "zc_verify")
    return bool(acc.value)


def prove_sumcheck_static(gate, n, d, cols, proof_out, roots=None, stream=None) -> None:
    """zc_prove_sumcheck_static: SumCheck proof with no device allocation.

    cols: CUDA tensors on the current device; proof_out: a CUDA uint8 tensor
    of at least proof_size(...) bytes.  Asynchronous on ``stream``.  For
    callers that may not allocate device memory while proving; the library's
    fixed static scratch (32 MiB) bounds the instance size."""
    p = zc_params(gate, n, d, 0)
    P = _Ptrs(cols)
    rb, rp = _roots_arg(roots)
    ln = ctypes.c_size_t()
    st = lib().zc_prove_sumcheck_static(ctypes.byref(p), P.p, rp, _stream_ptr(stream),
                                        _addr(proof_out), proof_out.numel(), ctypes.byref(ln))
    if st != ZC_OK:
        raise ZCError(st, "zc_prove_sumcheck_static")


# ---------------------------------------------------- commitment around it

def pcs_proof_size(n: int, c: int, t: int, nc: int = 0) -> int:
    out = ctypes.c_size_t()
    p = zc_pcs_params(n, nc, c, t)
    st = lib().zc_pcs_proof_size(ctypes.byref(p), ctypes.byref(out))
    if st != ZC_OK:
        raise ZCError(st, "zc_pcs_proof_size")
    return int(out.value)


def _bytes_array(items, count) -> np.ndarray:
    b = b"".join(bytes(x) for x in items)
    if len(b) != 32 * count:
        raise ValueError(f"expected {count} elements of 32 bytes")
    return np.frombuffer(b, dtype=np.uint8).copy()


class PcsCommitment:
    """zc_pcs handle: the encoded columns on the device and the Merkle tree."""

    def __init__(self, ctx: "Context", n: int, cols, t: int, nc: int = 0, stream=None):
        self.ctx = ctx
        self.n, self.c, self.t, self.nc = n, len(cols), t, nc
        P, on_dev = ctx._cols(cols)
        self._keep = (P, cols)
        p = zc_pcs_params(n, nc, self.c, t)
        h = ctypes.c_void_p()
        root = np.zeros(32, np.uint8)
        st = lib().zc_pcs_commit(ctx.h, ctypes.byref(p), P.p, on_dev, _stream_ptr(stream), ctypes.byref(h),
                                 root.ctypes.data)
        ctx._check(st, "zc_pcs_commit")
        self.h = h
        self.root = root.tobytes()

    def open(self, alpha, values, stream=None) -> bytes:
        a = _bytes_array(alpha, self.n)
        v = _bytes_array(values, self.c)
        cap = pcs_proof_size(self.n, self.c, self.t, self.nc)
        out = np.zeros(cap, np.uint8)
        ln = ctypes.c_size_t()
        st = lib().zc_pcs_open(self.h, a.ctypes.data, v.ctypes.data, _stream_ptr(stream),
                               out.ctypes.data, cap, ctypes.byref(ln))
        self.ctx._check(st, "zc_pcs_open")
        return out.tobytes()[: ln.value]

    def close(self):
        if getattr(self, "h", None):
            lib().zc_pcs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pcs_verify(n: int, c: int, t: int, root: bytes, alpha, values, proof, nc: int = 0) -> bool:
    """Host verifier of an opening (no GPU needed)."""
    p = zc_pcs_params(n, nc, c, t)
    a = _bytes_array(alpha, n)
    v = _bytes_array(values, c)
    r = np.frombuffer(bytes(root), dtype=np.uint8).copy()
    pr = _host_array(proof)
    acc = ctypes.c_int(0)
    st = lib().zc_pcs_verify(ctypes.byref(p), r.ctypes.data, a.ctypes.data,
                             v.ctypes.data, pr.ctypes.data, pr.size,
                             ctypes.byref(acc))
    if st == ZC_ERR_ARG:
        return False
    if st != ZC_OK:
        raise ZCError(st, "zc_pcs_verify")
    return bool(acc.value)


def sumcheck_point(gate, n, d, form, roots, proof):
    """(alpha, values, rounds_ok) of a SumCheck-form proof, replayed on the host."""
    p = zc_params(gate, n, d, 0)
    c = len(roots)
    rb = _bytes_array(roots, c)
    pr = _host_array(proof)
    a = np.zeros(32 * n, np.uint8)
    v = np.zeros(32 * c, np.uint8)
    ok = ctypes.c_int(0)
    st = lib().zc_sumcheck_point(ctypes.byref(p), form, rb.ctypes.data,
                                 pr.ctypes.data, pr.size, a.ctypes.data,
                                 v.ctypes.data, ctypes.byref(ok))
    if st != ZC_OK:
        raise ZCError(st, "zc_sumcheck_point")
    return ([a[32 * i:32 * i + 32].tobytes() for i in range(n)],
            [v[32 * j:32 * j + 32].tobytes() for j in range(c)], bool(ok.value))
