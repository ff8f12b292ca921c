"""The C ABI library loads, exports what include/zc.h declares, and its host
verifier agrees with the oracle (CPU only; no kernel is launched)."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2606_16146_gb300 import build, witness
from paper_2606_16146_gb300 import zc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "zc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(zc_[a-z_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    L = zc.lib(path)
    names = declared_functions()
    assert "zc_prove_sumcheck" in names and "zc_prove_ntt" in names and "zc_verify" in names
    for name in names:
        assert hasattr(L, name), name


@pytest.mark.parametrize("gate,n,d", [(1, 5, 3), (2, 7, 2), (2, 3, 32), (1, 24, 3), (3 | 3 << 8, 9, 2), (3, 6, 4)])
def test_proof_size_matches_oracle(gate, n, d):
    for form in (1, 2):
        assert zc.proof_size(gate, n, d, form) == oracle.proof_size(form, gate, n, d)


def test_bad_params_rejected():
    with pytest.raises(zc.ZCError):
        zc.proof_size(1, 5, 4, 1)          # Plonk needs d = 3
    with pytest.raises(zc.ZCError):
        zc.proof_size(2, 0, 2, 1)          # n >= 1
    with pytest.raises(zc.ZCError):
        zc.proof_size(4, 5, 3, 1)          # unknown gate
    with pytest.raises(zc.ZCError):
        zc.proof_size(zc.gate_sum(0), 5, 1, 1)   # sum gate needs a product of >= 2
    with pytest.raises(zc.ZCError):
        zc.proof_size(zc.gate_sum(60), 5, 8, 1)  # more than 65 columns
    with pytest.raises(zc.ZCError):
        zc.proof_size(2 | (1 << 8), 5, 3, 1)     # only the sum gate carries m


def test_setup_fails_loudly_without_a_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(zc.ZCError):
        zc.Context(0, 12, 3)


@pytest.mark.parametrize("gate,n,d", [(1, 6, 3), (2, 5, 4), (2, 1, 2), (1, 1, 3),
                                      (zc.gate_sum(3), 5, 2), (zc.gate_sum(0), 4, 3)])
def test_host_verifier_agrees_with_oracle(gate, n, d):
    cols = witness.generate(gate, n, d, 40 + n)
    bad = witness.generate(gate, n, d, 40 + n, tamper=True)
    ps = oracle.prove_sumcheck(gate, n, d, cols)
    assert zc.verify(gate, n, d, 1, cols, ps)
    assert not zc.verify(gate, n, d, 1, bad, oracle.prove_sumcheck(gate, n, d, bad))
    x = bytearray(ps)
    x[40] ^= 4
    assert not zc.verify(gate, n, d, 1, cols, bytes(x))
    pn, q = oracle.prove_ntt(gate, n, d, cols)
    assert zc.verify(gate, n, d, 2, cols, pn, q=q)
    pb, qb = oracle.prove_ntt(gate, n, d, bad)
    assert not zc.verify(gate, n, d, 2, bad, pb, q=qb)
    q2 = np.array(q, copy=True)
    q2[-1] ^= 1                      # top coefficient: breaks root and degree bound
    assert not zc.verify(gate, n, d, 2, cols, pn, q=q2)
    roots = [oracle.root(c) for c in cols]
    assert zc.verify(gate, n, d, 1, cols, ps, roots=roots)


@pytest.mark.parametrize("gate,n,d,ks", [(2, 5, 4, (1, 0)), (1, 7, 3, (1, 0)), (2, 3, 6, (2, 0)),
                                         (2, 4, 7, (2, 1)), (zc.gate_sum(1), 6, 3, (1, 0))])
def test_host_verifier_step_radix_domain(gate, n, d, ks):
    """The library's host verifier (its own Merkle root over 2^k N + 2^s N
    coefficients and its own header decoding) accepts the oracle's step-radix
    proofs and rejects a flipped quotient coefficient or a wrong domain word."""
    w = zc.domain_word(*ks)
    assert zc.domain_size(n, d, w) == oracle.domain_size(n, d, w)
    cols = witness.generate(gate, n, d, 60 + n)
    pn, q = oracle.prove_ntt(gate, n, d, cols, log_blowup=w)
    assert zc.verify(gate, n, d, 2, cols, pn, q=q, log_blowup=w)
    q2 = np.array(q, copy=True)
    q2[32 * 3] ^= 1
    assert not zc.verify(gate, n, d, 2, cols, pn, q=q2, log_blowup=w)
    # the header names another domain than the caller's: malformed, not accepted
    assert not zc.verify(gate, n, d, 2, cols, pn, q=q, log_blowup=ks[0] + 1)


@pytest.mark.parametrize("gate,n,d", [(1, 6, 3), (2, 5, 4), (2, 1, 2), (zc.gate_sum(2), 4, 3)])
def test_host_verifier_eq_factored(gate, n, d):
    """ZC_FORM_SUMCHECK_EQ: the library's host verifier accepts the oracle's
    eq-factored proofs, rejects tampered ones, and sizes them as the oracle."""
    assert zc.proof_size(gate, n, d, zc.ZC_FORM_SUMCHECK_EQ) == oracle.proof_size_eq(gate, n, d)
    cols = witness.generate(gate, n, d, 90 + n)
    pb = oracle.prove_sumcheck_eq(gate, n, d, cols)
    assert zc.verify(gate, n, d, zc.ZC_FORM_SUMCHECK_EQ, cols, pb)
    assert not zc.verify(gate, n, d, zc.ZC_FORM_SUMCHECK, cols, pb)
    bad = witness.generate(gate, n, d, 90 + n, tamper=True)
    assert not zc.verify(gate, n, d, zc.ZC_FORM_SUMCHECK_EQ, bad, oracle.prove_sumcheck_eq(gate, n, d, bad))
    x = bytearray(pb)
    x[16 + 32 * (d + 1) + 1] ^= 8
    assert not zc.verify(gate, n, d, zc.ZC_FORM_SUMCHECK_EQ, cols, bytes(x))


@pytest.mark.parametrize("n,nc,gate,d", [(4, 2, 1, 3), (5, 5, 2, 3), (6, 3, 2, 2)])
def test_host_pcs_verifier_and_sumcheck_point(n, nc, gate, d):
    """The library's host side of the commitment: zc_sumcheck_point replays
    an oracle SumCheck proof (PCS root as every column root) to the oracle's
    alpha and final values, and zc_pcs_verify accepts the oracle's opening
    there and rejects a flipped byte or a wrong value."""
    cols = witness.generate(gate, n, d, 130 + n)
    c, t = len(cols), 7
    root = oracle.pcs_commit(n, cols, nc=nc)
    for form in (zc.ZC_FORM_SUMCHECK, zc.ZC_FORM_SUMCHECK_EQ):
        prove = oracle.prove_sumcheck if form == zc.ZC_FORM_SUMCHECK else oracle.prove_sumcheck_eq
        pb, _, al = prove(gate, n, d, cols, roots=[root] * c, with_challenges=True)
        alpha, vals, ok = zc.sumcheck_point(gate, n, d, form, [root] * c, pb)
        assert ok and alpha == al
        assert vals == [pb[len(pb) - 32 * (c - j):len(pb) - 32 * (c - j) + 32] for j in range(c)]
        pr = oracle.pcs_open(n, cols, alpha, vals, t, nc=nc)
        assert len(pr) == zc.pcs_proof_size(n, c, t, nc)
        assert zc.pcs_verify(n, c, t, root, alpha, vals, pr, nc)
        x = bytearray(pr)
        x[len(pr) // 2] ^= 1
        assert not zc.pcs_verify(n, c, t, root, alpha, vals, bytes(x), nc)
        v2 = list(vals)
        v2[0] = bytes([vals[0][0] ^ 1]) + vals[0][1:]
        assert not zc.pcs_verify(n, c, t, root, alpha, v2, pr, nc)
    bad = bytearray(pb)
    bad[20] ^= 1
    assert not zc.sumcheck_point(gate, n, d, zc.ZC_FORM_SUMCHECK_EQ, [root] * c, bytes(bad))[2]
