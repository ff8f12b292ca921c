"""Pins the CPU oracle to things other than itself (CPU only).

Field ops against Python integers, SHA-256 against hashlib and the FIPS 180-4
examples, transforms against O(N^2) DFTs and Horner evaluation, quotients
against schoolbook long division by x^N - 1 (Sec. 3.2), SumCheck round
polynomials against their brute-force definition (Fig. side-by-side-zc,
right) and the final values against direct MLE evaluation (Sec. 3.3).
"""
import os
import random

import numpy as np
import pytest

import mini_zc as mz
import oracle
from paper_2606_16146_gb300 import witness

R = mz.R
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_golden_modulus_facts():
    kv = dict(line.split() for line in open(os.path.join(GOLDEN, "bls12_381_fr.txt")))
    r = int(kv["r"], 16)
    assert r == R
    s = int(kv["two_adicity"])
    assert (r - 1) % (1 << s) == 0 and ((r - 1) >> s) % 2 == 1
    g = int(kv["generator"])
    assert pow(g, (r - 1) // 2, r) == r - 1          # quadratic non-residue
    w = pow(g, (r - 1) >> s, r)
    assert oracle.root_of_unity(32) == w


EDGES = [0, 1, 2, R - 1, R - 2, (1 << 255) % R, (1 << 256) % R, (1 << 254), R // 2, R // 2 + 1]


@pytest.mark.parametrize("op", ["add", "sub", "mul"])
def test_field_binary_ops(op):
    rng = random.Random(11)
    vals = EDGES + [rng.randrange(R) for _ in range(60)]
    ref = {"add": lambda a, b: (a + b) % R, "sub": lambda a, b: (a - b) % R,
           "mul": lambda a, b: a * b % R}[op]
    for a in vals[:30]:
        for b in vals[::3]:
            assert oracle.fr(op, a, b) == ref(a, b), (op, a, b)


def test_field_unary_ops():
    rng = random.Random(12)
    for a in EDGES[1:] + [rng.randrange(1, R) for _ in range(40)]:
        assert oracle.fr("inv", a) * a % R == 1
        assert oracle.fr("neg", a) == (-a) % R
    with pytest.raises(ValueError):
        oracle.fr("inv", 0)
    with pytest.raises(ValueError):
        oracle.fr("add", R, 1)                     # non-canonical input rejected


def test_sha256_fips_examples():
    for line in open(os.path.join(GOLDEN, "sha256_fips180.txt")):
        m, h = line.rstrip("\n").split(" ")
        assert oracle.sha256(bytes.fromhex(m)).hex() == h


def test_sha256_against_hashlib():
    import hashlib
    rng = random.Random(3)
    for ln in list(range(0, 200)) + [447, 448, 511, 512, 1000, 4096, 4097]:
        m = bytes(rng.randrange(256) for _ in range(ln))
        assert oracle.sha256(m) == hashlib.sha256(m).digest()


@pytest.mark.parametrize("logn", [1, 2, 5, 11, 20, 32])
def test_roots_of_unity(logn):
    w = oracle.root_of_unity(logn)
    assert pow(w, 1 << logn, R) == 1
    assert pow(w, 1 << (logn - 1), R) == R - 1       # primitive: w^(N/2) = -1


@pytest.mark.parametrize("logn", [0, 1, 2, 3, 4, 5, 6])
def test_ntt_matches_dft(logn):
    rng = random.Random(100 + logn)
    N = 1 << logn
    a = [rng.randrange(R) for _ in range(N)]
    assert oracle.ntt(a, logn) == mz.dft(a, mz.omega(logn))
    coef = oracle.ntt(a, logn, inverse=True)
    assert coef == mz.interpolate_h(a)
    assert oracle.ntt(coef, logn) == a               # round trip


def test_ntt_roundtrip_large():
    rng = np.random.default_rng(5)
    logn = 12
    a = [int(x) % R for x in rng.integers(0, 2**62, size=1 << logn)]
    assert oracle.ntt(oracle.ntt(a, logn, inverse=True), logn) == a


@pytest.mark.parametrize("n,logm", [(1, 1), (2, 4), (3, 5), (4, 6), (5, 7)])
def test_coset_lde_matches_horner(n, logm):
    rng = random.Random(7 * n + logm)
    coef = [rng.randrange(R) for _ in range(1 << n)]
    out = oracle.coset_lde(coef, n, logm)
    w = mz.omega(logm)
    for i in range(1 << logm):
        assert out[i] == mz.horner(coef, 7 * pow(w, i, R) % R)


@pytest.mark.parametrize("L", [1, 2, 32, 64, 128, 1024])
def test_merkle_root(L):
    rng = random.Random(L)
    v = [rng.randrange(R) for _ in range(L)]
    assert oracle.root(oracle.ints_to_bytes(v)) == mz.merkle_root(v)


def test_transcript_bytes():
    m = bytes(range(77))
    t = mz.Transcript(1, 1, 5, 3, 0)
    t.absorb(m)
    assert oracle.transcript_demo(1, 1, 5, 3, 0, m) == t.squeeze()


def _cols_int(cols):
    return [mz.ints(c) for c in cols]


# the paper's workload family (Table poly_examples) as sum gates: gate word, d
FAMILY = [(witness.gate_sum(0), 2), (witness.gate_sum(1), 2), (witness.gate_sum(2), 2),
          (witness.gate_sum(3), 2), (witness.gate_sum(0), 3), (witness.gate_sum(0), 4)]

SC_CASES = [(1, 1, 3), (1, 2, 3), (1, 3, 3), (1, 4, 3), (2, 1, 2), (2, 3, 2), (2, 3, 3), (2, 2, 5), (2, 4, 4)]
SC_CASES += [(g, n, d) for (g, d), n in zip(FAMILY, (1, 3, 2, 3, 3, 2))]


@pytest.mark.parametrize("gate,n,d", SC_CASES)
def test_sumcheck_proof_matches_bruteforce(gate, n, d):
    cols = witness.generate(gate, n, d, 77 + n + d)
    pb, r, al = oracle.prove_sumcheck(gate, n, d, cols, with_challenges=True)
    ref, r2, al2 = mz.prove_sumcheck(gate, n, d, _cols_int(cols))
    assert [int.from_bytes(x, "little") for x in r] == r2
    assert [int.from_bytes(x, "little") for x in al] == al2
    assert pb == ref


@pytest.mark.parametrize("gate,n,d", [(1, 3, 3), (2, 3, 4), (witness.gate_sum(2), 3, 2),
                                      (witness.gate_sum(0), 2, 3)])
def test_sumcheck_tampered_matches_bruteforce(gate, n, d):
    cols = witness.generate(gate, n, d, 91, tamper=True)
    pb = oracle.prove_sumcheck(gate, n, d, cols)
    ref, _, _ = mz.prove_sumcheck(gate, n, d, _cols_int(cols))
    assert pb == ref


def test_sumcheck_round_degree_bound():
    """G_i has degree <= d+1: the brute-force value at t = d+2 equals the
    extrapolation of the d+2 values in the proof."""
    gate, n, d = 2, 3, 3
    cols = witness.generate(gate, n, d, 5)
    ci = _cols_int(cols)
    pb, r, al = oracle.prove_sumcheck(gate, n, d, cols, with_challenges=True)
    r = [int.from_bytes(x, "little") for x in r]
    al = [int.from_bytes(x, "little") for x in al]
    G = mz.ints(pb[16:16 + 32 * n * (d + 2)])
    for i in range(n):
        g = G[i * (d + 2):(i + 1) * (d + 2)]
        x = d + 2
        ext = 0
        for t in range(d + 2):
            num = den = 1
            for s in range(d + 2):
                if s != t:
                    num = num * (x - s) % R
                    den = den * (t - s) % R
            ext = (ext + g[t] * num * mz.inv(den)) % R
        assert ext == mz.sumcheck_round_poly(gate, d, ci, r, al, i, x)


def test_sumcheck_round_invariant_and_final():
    gate, n, d = 1, 6, 3
    cols = witness.generate(gate, n, d, 1006)
    pb, r, al = oracle.prove_sumcheck(gate, n, d, cols, with_challenges=True)
    r = [int.from_bytes(x, "little") for x in r]
    al = [int.from_bytes(x, "little") for x in al]
    G = mz.ints(pb[16:16 + 32 * n * (d + 2)])
    claim = 0
    for i in range(n):
        g = G[i * (d + 2):(i + 1) * (d + 2)]
        assert (g[0] + g[1]) % R == claim
        claim = 0
        for t in range(d + 2):
            num = den = 1
            for s in range(d + 2):
                if s != t:
                    num = num * (al[i] - s) % R
                    den = den * (t - s) % R
            claim = (claim + g[t] * num * mz.inv(den)) % R
    v = mz.ints(pb[16 + 32 * n * (d + 2):])
    ci = _cols_int(cols)
    for j in range(8):
        assert v[j] == mz.mle(ci[j], al)
    assert claim == mz.gate_eval(gate, d, v) * mz.eq(r, al) % R


NTT_CASES = [(1, 1, 3), (1, 2, 3), (1, 3, 3), (1, 5, 3), (2, 1, 2), (2, 3, 2), (2, 2, 3), (2, 3, 4), (2, 2, 5), (2, 4, 8)]
NTT_CASES += [(g, n, d) for (g, d), n in zip(FAMILY, (2, 1, 3, 2, 3, 2))]


@pytest.mark.parametrize("gate,n,d", NTT_CASES)
def test_ntt_proof_matches_long_division(gate, n, d):
    cols = witness.generate(gate, n, d, 300 + n * d)
    pb, q = oracle.prove_ntt(gate, n, d, cols)
    ref, qref, z = mz.prove_ntt(gate, n, d, _cols_int(cols))
    assert mz.ints(q) == qref
    assert pb == ref


@pytest.mark.parametrize("gate,n,d", [(1, 3, 3), (1, 5, 3), (2, 4, 3), (witness.gate_sum(0), 3, 3),
                                      (witness.gate_sum(1), 4, 3)])
def test_ntt_quotient_sized_domain_matches_long_division(gate, n, d):
    # |D| = 2N for degree 3: the quotient's (d-1)N - d + 1 coefficients fit (Sec. 4)
    cols = witness.generate(gate, n, d, 350 + n * d)
    pb, q = oracle.prove_ntt(gate, n, d, cols, log_blowup=1)
    ref, qref, _ = mz.prove_ntt(gate, n, d, _cols_int(cols), logb=1)
    assert mz.ints(q) == qref
    assert pb == ref
    assert oracle.verify_ntt(gate, n, d, cols, pb, q)


def test_ntt_domain_below_the_quotient_rejected():
    cols = witness.generate(2, 3, 4, 7)
    with pytest.raises(Exception):
        oracle.prove_ntt(2, 3, 4, cols, log_blowup=1)   # 2N < 3N - 3


def test_ntt_quotient_degree_and_identity():
    gate, n, d = 1, 8, 3
    cols = witness.generate(gate, n, d, 1008)
    pb, q = oracle.prove_ntt(gate, n, d, cols)
    qi = mz.ints(q)
    N = 1 << n
    qlen = (d - 1) * N - d + 1
    assert all(x == 0 for x in qi[qlen:])
    assert qi[qlen - 1] != 0
    coefs = [mz.interpolate_h(c) for c in _cols_int(cols)]
    rng = random.Random(1)
    for _ in range(3):
        z = rng.randrange(R)
        ys = [mz.horner(cf, z) for cf in coefs]
        assert mz.gate_eval(gate, d, ys) == mz.horner(qi, z) * (pow(z, N, R) - 1) % R


def test_ntt_tampered_quotient_interpolates_on_coset():
    """For a witness that does not vanish on H, q is the degree < M
    interpolant of f/z_H on D (Fig. side-by-side-zc, left, lines INTT_D)."""
    gate, n, d = 1, 3, 3
    cols = witness.generate(gate, n, d, 44, tamper=True)
    pb, q = oracle.prove_ntt(gate, n, d, cols)
    qi = mz.ints(q)
    N, M = 1 << n, 1 << (n + 2)
    coefs = [mz.interpolate_h(c) for c in _cols_int(cols)]
    w = mz.omega(n + 2)
    for i in range(M):
        x = 7 * pow(w, i, R) % R
        f = mz.gate_eval(gate, d, [mz.horner(cf, x) for cf in coefs])
        assert mz.horner(qi, x) == f * mz.inv(pow(x, N, R) - 1) % R
    assert any(qi[(d - 1) * N - d + 1:])            # degree bound broken


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("gate,n,d", [(1, 7, 3), (2, 6, 4), (witness.gate_sum(1), 6, 2),
                                      (witness.gate_sum(0), 5, 4)])
def test_verifier_accepts_honest_rejects_tampered(form, gate, n, d):
    cols = witness.generate(gate, n, d, 500 + n)
    bad = witness.generate(gate, n, d, 500 + n, tamper=True)
    if form == 1:
        pb = oracle.prove_sumcheck(gate, n, d, cols)
        assert oracle.verify_sumcheck(gate, n, d, cols, pb)
        pbad = oracle.prove_sumcheck(gate, n, d, bad)
        assert not oracle.verify_sumcheck(gate, n, d, bad, pbad)
        # a proof for the honest columns does not verify against other columns
        assert not oracle.verify_sumcheck(gate, n, d, bad, pb)
        for off in (16, 16 + 32 * 5, len(pb) - 32):
            x = bytearray(pb)
            x[off] ^= 1
            assert not oracle.verify_sumcheck(gate, n, d, cols, bytes(x))
    else:
        pb, q = oracle.prove_ntt(gate, n, d, cols)
        assert oracle.verify_ntt(gate, n, d, cols, pb, q)
        pbad, qbad = oracle.prove_ntt(gate, n, d, bad)
        assert not oracle.verify_ntt(gate, n, d, bad, pbad, qbad)
        for off in (20, 52, len(pb) - 32):
            x = bytearray(pb)
            x[off] ^= 1
            assert not oracle.verify_ntt(gate, n, d, cols, bytes(x), q)
        q2 = np.array(q, copy=True)
        q2[0] ^= 1
        assert not oracle.verify_ntt(gate, n, d, cols, pb, q2)


def test_witness_generator_satisfies_gate():
    for gate, n, d in [(1, 5, 3), (2, 5, 2), (2, 4, 7)] + [(g, 5, d) for g, d in FAMILY]:
        cols = _cols_int(witness.generate(gate, n, d, 9))
        for k in range(1 << n):
            assert mz.gate_eval(gate, d, [c[k] for c in cols]) == 0
        bad = _cols_int(witness.generate(gate, n, d, 9, tamper=True))
        viol = [k for k in range(1 << n) if mz.gate_eval(gate, d, [c[k] for c in bad]) != 0]
        assert viol == [9 % (1 << n)]


EDGE_CASES = [(1, 2, 3), (1, 3, 3), (2, 3, 2), (2, 2, 4), (witness.gate_sum(2), 2, 2), (witness.gate_sum(0), 3, 3)]


@pytest.mark.parametrize("gate,n,d", EDGE_CASES)
def test_edge_value_inputs_match_bruteforce(gate, n, d):
    """Boundary field values (0, 1, r-1, r-2^k, 2^k, ...), gate not satisfied:
    both oracle provers still equal the big-integer restatement."""
    cols = witness.generate_edge(gate, n, d, 4242 + n, only_edges=True)
    ci = _cols_int(cols)
    assert all(v < R for c in ci for v in c)
    ref, _, _ = mz.prove_sumcheck(gate, n, d, ci)
    assert oracle.prove_sumcheck(gate, n, d, cols) == ref
    pb, q = oracle.prove_ntt(gate, n, d, cols)
    refn, qref, _ = mz.prove_ntt(gate, n, d, ci)
    assert mz.ints(q) == qref
    assert pb == refn


def test_edge_witness_covers_the_boundaries():
    vals = {v for c in _cols_int(witness.generate_edge(2, 8, 4, 1, only_edges=True)) for v in c}
    for v in (0, 1, 2, R - 1, R - 2, R - 3, 2**254, R - 2**254, 2**32 - 1, R - 2**32, (R - 1) // 2,
              (R + 1) // 2, 2**256 % R, 2**512 % R):
        assert v in vals, hex(v)
    mixed = _cols_int(witness.generate_edge(1, 8, 3, 1))
    assert any(v not in vals for c in mixed for v in c)


# ---- step-radix NTT domain (Sec. 4, "Degree scaling": 3N = 2N + N, 5N = 4N + N)

STEP_CASES = [(1, 3, 3, (1, 0)), (2, 3, 4, (1, 0)), (2, 2, 6, (2, 0)), (2, 3, 7, (2, 1)),
              (2, 2, 3, (1, 0)), (witness.gate_sum(1), 3, 4, (1, 0)), (witness.gate_sum(0), 2, 4, (1, 0))]


@pytest.mark.parametrize("gate,n,d,ks", STEP_CASES)
def test_ntt_step_radix_matches_long_division(gate, n, d, ks):
    """Honest witness on a 2^k N + 2^s N domain: the quotient is the long
    division of f by x^N - 1, padded to M; proof bytes as the restatement."""
    cols = witness.generate(gate, n, d, 500 + n * d)
    w = oracle.domain_word(*ks)
    pb, q = oracle.prove_ntt(gate, n, d, cols, log_blowup=w)
    ref, qref, _ = mz.prove_ntt(gate, n, d, _cols_int(cols), logb=ks)
    assert len(qref) == oracle.domain_size(n, d, w) == ((1 << ks[0]) + (1 << ks[1])) << n
    assert mz.ints(q) == qref
    assert pb == ref
    assert oracle.verify_ntt(gate, n, d, cols, pb, q)


@pytest.mark.parametrize("gate,n,d,ks", [(1, 2, 3, (1, 0)), (2, 2, 4, (1, 0)), (2, 1, 6, (2, 0)),
                                         (2, 2, 5, (2, 1))])
def test_ntt_step_radix_interpolates_nonvanishing(gate, n, d, ks):
    """Witness that does not vanish on H: q is the degree < M interpolant of
    f / z_H on the M explicit points of D_big u D_small (Lagrange)."""
    cols = witness.generate_edge(gate, n, d, 77 + n)
    w = oracle.domain_word(*ks)
    pb, q = oracle.prove_ntt(gate, n, d, cols, log_blowup=w)
    ref, qref, _ = mz.prove_ntt(gate, n, d, _cols_int(cols), logb=ks)
    assert mz.ints(q) == qref
    assert pb == ref


def test_ntt_step_radix_identity_and_rejections():
    gate, n, d = 2, 6, 4
    cols = witness.generate(gate, n, d, 61)
    w = oracle.domain_word(1, 0)                      # 3N
    pb, q = oracle.prove_ntt(gate, n, d, cols, log_blowup=w)
    qi = mz.ints(q)
    N = 1 << n
    qlen = (d - 1) * N - d + 1
    assert len(qi) == 3 * N and all(x == 0 for x in qi[qlen:]) and qi[qlen - 1] != 0
    coefs = [mz.interpolate_h(c) for c in _cols_int(cols)]
    rng = random.Random(5)
    for _ in range(3):
        z = rng.randrange(R)
        ys = [mz.horner(cf, z) for cf in coefs]
        assert mz.gate_eval(gate, d, ys) == mz.horner(qi, z) * (pow(z, N, R) - 1) % R
    # same quotient polynomial as the power-of-two 4N domain, other bytes
    pb4, q4 = oracle.prove_ntt(gate, n, d, cols)
    assert mz.ints(q4)[:3 * N] == qi and pb4 != pb
    # tampered witness or quotient: rejected
    bad = witness.generate(gate, n, d, 61, tamper=True)
    pbb, qb = oracle.prove_ntt(gate, n, d, bad, log_blowup=w)
    assert not oracle.verify_ntt(gate, n, d, bad, pbb, qb)
    q2 = np.array(q, copy=True)
    q2[32 * 5] ^= 1
    assert not oracle.verify_ntt(gate, n, d, cols, pb, q2)
    # domains that cannot hold q, or malformed words
    with pytest.raises(ValueError):
        oracle.prove_ntt(2, 4, 6, witness.generate(2, 4, 6, 1), log_blowup=oracle.domain_word(1, 0))
    with pytest.raises(ValueError):
        oracle.prove_ntt(gate, n, d, cols, log_blowup=oracle.domain_word(1, 1))   # s must be < k


@pytest.mark.parametrize("L", [1, 3, 5, 63, 64, 65, 96, 100, 192, 200, 3 * 1024, 5 * 512 + 64])
def test_merkle_root_any_length(L):
    rng = random.Random(L)
    vals = [rng.randrange(R) for _ in range(L)]
    assert oracle.root(oracle.ints_to_bytes(vals)) == mz.merkle_root(vals)


# ---- eq-factored SumCheck, transcript v2 (rounds carry H_i(0..d))

EQ_CASES = [(1, 1, 3), (1, 3, 3), (2, 3, 2), (2, 2, 5), (2, 3, 4), (witness.gate_sum(1), 3, 2),
            (witness.gate_sum(0), 2, 3)]


@pytest.mark.parametrize("gate,n,d", EQ_CASES)
def test_sumcheck_eq_matches_bruteforce(gate, n, d):
    cols = witness.generate(gate, n, d, 700 + n + d)
    pb, r, al = oracle.prove_sumcheck_eq(gate, n, d, cols, with_challenges=True)
    ref, r2, al2 = mz.prove_sumcheck_eq(gate, n, d, _cols_int(cols))
    assert [int.from_bytes(x, "little") for x in r] == r2
    assert [int.from_bytes(x, "little") for x in al] == al2
    assert pb == ref
    assert len(pb) == oracle.proof_size_eq(gate, n, d) == 16 + 32 * (n * (d + 1) + len(cols))


def test_sumcheck_eq_is_g_with_the_eq_factor_split_off():
    """G_i(t) (brute force, v1 definition) = c_i l_i(t) H_i(t) at the v2
    proof's own challenges, c_i = prod_{j<i} eq(alpha_j, r_j)."""
    gate, n, d = 2, 3, 3
    cols = witness.generate(gate, n, d, 17)
    ci = _cols_int(cols)
    pb, r, al = oracle.prove_sumcheck_eq(gate, n, d, cols, with_challenges=True)
    r = [int.from_bytes(x, "little") for x in r]
    al = [int.from_bytes(x, "little") for x in al]
    H = mz.ints(pb[16:16 + 32 * n * (d + 1)])
    for i in range(n):
        c = 1
        for j in range(i):
            c = c * ((1 - r[j]) * (1 - al[j]) + r[j] * al[j]) % R
        for t in range(d + 2):
            li = ((1 - r[i]) * (1 - t) + r[i] * t) % R
            g = mz.sumcheck_round_poly(gate, d, ci, r, al, i, t)
            h = H[i * (d + 1) + t] if t <= d else mz.sumcheck_round_h(gate, d, ci, r, al, i, t)
            assert g == c * li * h % R


@pytest.mark.parametrize("gate,n,d", [(1, 6, 3), (2, 5, 4), (witness.gate_sum(2), 5, 2)])
def test_sumcheck_eq_verifier(gate, n, d):
    cols = witness.generate(gate, n, d, 800 + n)
    pb = oracle.prove_sumcheck_eq(gate, n, d, cols)
    assert oracle.verify_sumcheck_eq(gate, n, d, cols, pb)
    assert not oracle.verify_sumcheck(gate, n, d, cols, pb)          # not a v1 proof
    bad = witness.generate(gate, n, d, 800 + n, tamper=True)
    assert not oracle.verify_sumcheck_eq(gate, n, d, bad, oracle.prove_sumcheck_eq(gate, n, d, bad))
    for off in (16, 16 + 32 * (d + 1) + 5, len(pb) - 3):
        x = bytearray(pb)
        x[off] ^= 2
        assert not oracle.verify_sumcheck_eq(gate, n, d, cols, bytes(x))


# ---- hash-based PCS (Ligero-style) around the ZeroCheck




def _sc_point(gate, n, d, cols, root):
    pb, r, al = oracle.prove_sumcheck(gate, n, d, cols, roots=[root] * len(cols), with_challenges=True)
    c = len(cols)
    vals = [pb[len(pb) - 32 * (c - j):len(pb) - 32 * (c - j) + 32] for j in range(c)]
    return pb, al, vals


@pytest.mark.parametrize("gate,n,nc,d", [(g, n, nc, d) for g, n, nc, d in
                                         [(1, 3, 2, 3), (2, 4, 2, 2), (2, 5, 3, 3), (witness.gate_sum(1), 4, 4, 2)]])
def test_pcs_matches_restatement(gate, n, nc, d):
    """Commitment root and opening bytes (u_j, u', queried columns, Merkle
    paths) equal the big-integer restatement; the opening's u_j reproduce the
    columns' MLE values at alpha (Sec. 3.3 interpolation form)."""
    cols = witness.generate(gate, n, d, 1200 + n)
    ci = _cols_int(cols)
    root = oracle.pcs_commit(n, cols, nc=nc)
    pb, al, vals = _sc_point(gate, n, d, cols, root)
    t = 5
    pr = oracle.pcs_open(n, cols, al, vals, t, nc=nc)
    alpha = [int.from_bytes(a, "little") for a in al]
    ref, rroot, us = mz.pcs_open(n, nc, ci, alpha, [int.from_bytes(v, "little") for v in vals], t)
    assert root == rroot
    assert pr == ref
    el = mz.eq_tab(alpha[n - nc:])
    for j, col in enumerate(ci):
        mle = mz.mle(col, alpha)
        assert mle == int.from_bytes(vals[j], "little")
        assert sum(u * e for u, e in zip(us[j], el)) % R == mle
    assert oracle.pcs_verify(n, len(cols), t, root, al, vals, pr, nc=nc)


def test_pcs_rejections():
    gate, n, nc, d, t = 2, 6, 3, 3, 24
    cols = witness.generate(gate, n, d, 1300)
    root = oracle.pcs_commit(n, cols, nc=nc)
    pb, al, vals = _sc_point(gate, n, d, cols, root)
    pr = oracle.pcs_open(n, cols, al, vals, t, nc=nc)
    c = len(cols)
    assert oracle.pcs_verify(n, c, t, root, al, vals, pr, nc=nc)
    w, m = 1 << nc, 1 << (n - nc)
    off_u, off_up, off_q = 20, 20 + 32 * c * w, 20 + 32 * (c + 1) * w
    for off in (off_u + 7, off_up + 40, off_q + 3, off_q + 32 * c * m + 5, len(pr) - 1):
        x = bytearray(pr)
        x[off] ^= 1
        assert not oracle.pcs_verify(n, c, t, root, al, vals, bytes(x), nc=nc), off
    v2 = list(vals)
    v2[1] = bytes([vals[1][0] ^ 1]) + vals[1][1:]
    assert not oracle.pcs_verify(n, c, t, root, al, v2, pr, nc=nc)
    a2 = list(al)
    a2[0] = bytes([al[0][0] ^ 1]) + al[0][1:]
    assert not oracle.pcs_verify(n, c, t, root, a2, vals, pr, nc=nc)
    other = witness.generate(gate, n, d, 1301)
    assert not oracle.pcs_verify(n, c, t, oracle.pcs_commit(n, other, nc=nc), al, vals, pr, nc=nc)
    # the committed matrix of another witness cannot be opened to this one's values
    pr_o = oracle.pcs_open(n, other, al, vals, t, nc=nc)
    assert not oracle.pcs_verify(n, c, t, oracle.pcs_commit(n, other, nc=nc), al, vals, pr_o, nc=nc)
