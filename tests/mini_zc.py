"""Independent big-integer restatement of the ZeroCheck definitions, used to pin
the oracle on tiny inputs.

Everything here follows the mathematical definitions directly and shares
nothing with ``oracle/`` or the CUDA library: Python integers for the field,
``hashlib`` for SHA-256, O(N^2) DFTs, schoolbook polynomial products and long
division for the quotient (Sec. 3.2), and MLE evaluation by its interpolation
formula f~(x) = sum_b f(b) eq_x(b) (Sec. 3.3) for the SumCheck round
polynomials, with no folding.  Exponential or quadratic cost: tiny n only.
"""
from __future__ import annotations

import hashlib
import itertools
import math

R = 0x73eda753299d7d483339d80809a1d80553bda402fffe5bfeffffffff00000001
TAG = b"zerocheck-gb300/v1"


def inv(x):
    return pow(x, R - 2, R)


def omega(logn):
    return pow(pow(7, (R - 1) >> 32, R), 1 << (32 - logn), R)


def ints(buf) -> list[int]:
    b = bytes(buf)
    return [int.from_bytes(b[i:i + 32], "little") for i in range(0, len(b), 32)]


def enc(x) -> bytes:
    return int(x % R).to_bytes(32, "little")


def sha(m: bytes) -> bytes:
    return hashlib.sha256(m).digest()


def merkle_root(vals) -> bytes:
    """Leaves of 64 elements (the last may be shorter), pairwise SHA-256 up a
    binary tree whose odd last node moves up unchanged, then the length."""
    L = len(vals)
    nodes = [sha(b"".join(enc(v) for v in vals[i:i + 64])) for i in range(0, L, 64)]
    while len(nodes) > 1:
        nxt = [sha(nodes[2 * i] + nodes[2 * i + 1]) for i in range(len(nodes) // 2)]
        if len(nodes) % 2:
            nxt.append(nodes[-1])
        nodes = nxt
    return sha(L.to_bytes(8, "little") + nodes[0])


class Transcript:
    def __init__(self, form, gate, n, d, logm, tag=TAG):
        self.s = sha(tag + b"".join(x.to_bytes(4, "little") for x in (form, gate, n, d, logm)))

    def absorb(self, m: bytes):
        self.s = sha(self.s + m)

    def squeeze(self) -> int:
        self.s = sha(self.s + b"\x43")
        return int.from_bytes(self.s, "little") % R


def gate_eval(gate, d, x):
    if gate == 1:
        qL, qR, qM, qO, qC, a, b, c = x
        return (qL * a + qR * b + qM * a * b + qO * c + qC) % R
    if gate & 0xFF == 2:
        return (math.prod(x[:d]) - x[d]) % R
    return (math.prod(x[:d]) + sum(x[d:d + (gate >> 8)])) % R


# ---------------------------------------------------------------- MLE ---

def eq(x, b):
    """eq_x(b) = prod_i ((1-b_i)(1-x_i) + b_i x_i)"""
    p = 1
    for xi, bi in zip(x, b):
        p = p * ((1 - bi) * (1 - xi) + bi * xi) % R
    return p


def bits_msb(k, n):
    return [(k >> (n - 1 - i)) & 1 for i in range(n)]


def mle(table, x):
    """f~(x) = sum_b f(b) eq_x(b); b_1 is the most significant index bit."""
    n = len(x)
    return sum(table[k] * eq(x, bits_msb(k, n)) for k in range(1 << n)) % R


def sumcheck_round_poly(gate, d, cols, r, alphas, i, t):
    """G_i(t) = sum over x_{i+1..n} of f_M(a, t, x) eq_r(a, t, x)  (Fig. side-by-side-zc)."""
    n = len(r)
    tot = 0
    for rest in itertools.product((0, 1), repeat=n - i - 1):
        pt = list(alphas[:i]) + [t] + list(rest)
        vals = [mle(c, pt) for c in cols]
        tot += gate_eval(gate, d, vals) * eq(r, pt)
    return tot % R


def prove_sumcheck(gate, n, d, cols_int):
    c = len(cols_int)
    tr = Transcript(1, gate, n, d, 0)
    for col in cols_int:
        tr.absorb(merkle_root(col))
    r = [tr.squeeze() for _ in range(n)]
    out = b"ZCS1" + b"".join(x.to_bytes(4, "little") for x in (gate, n, d))
    alphas = []
    for i in range(n):
        G = [sumcheck_round_poly(gate, d, cols_int, r, alphas, i, t) for t in range(d + 2)]
        msg = b"".join(enc(g) for g in G)
        out += msg
        tr.absorb(msg)
        alphas.append(tr.squeeze())
    for col in cols_int:
        out += enc(mle(col, alphas))
    return out, r, alphas


def sumcheck_round_h(gate, d, cols, r, alphas, i, t):
    """H_i(t) = sum over x_{i+1..n} of f_M(a, t, x) eq_{r_{>i}}(x): G_i with the
    eq factors of the bound variables and of x_i itself divided out."""
    n = len(r)
    tot = 0
    for rest in itertools.product((0, 1), repeat=n - i - 1):
        pt = list(alphas[:i]) + [t] + list(rest)
        vals = [mle(c, pt) for c in cols]
        tot += gate_eval(gate, d, vals) * eq(r[i + 1:], rest)
    return tot % R


def prove_sumcheck_eq(gate, n, d, cols_int):
    """Eq-factored rounds ("ZCS2", tag v2): H_i at t = 0..d."""
    tr = Transcript(3, gate, n, d, 0, tag=b"zerocheck-gb300/v2")
    for col in cols_int:
        tr.absorb(merkle_root(col))
    r = [tr.squeeze() for _ in range(n)]
    out = b"ZCS2" + b"".join(x.to_bytes(4, "little") for x in (gate, n, d))
    alphas = []
    for i in range(n):
        H = [sumcheck_round_h(gate, d, cols_int, r, alphas, i, t) for t in range(d + 1)]
        msg = b"".join(enc(h) for h in H)
        out += msg
        tr.absorb(msg)
        alphas.append(tr.squeeze())
    for col in cols_int:
        out += enc(mle(col, alphas))
    return out, r, alphas


# ---------------------------------------------------------------- NTT ---

def dft(a, w):
    N = len(a)
    return [sum(a[k] * pow(w, i * k, R) for k in range(N)) % R for i in range(N)]


def interpolate_h(evals):
    """coefficients of the degree < N polynomial with g(w_N^i) = evals[i]"""
    N = len(evals)
    w = omega(N.bit_length() - 1)
    ninv = inv(N)
    return [x * ninv % R for x in dft(evals, inv(w))]


def horner(coef, x):
    acc = 0
    for cf in reversed(coef):
        acc = (acc * x + cf) % R
    return acc


def pmul(a, b):
    out = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        if x:
            for j, y in enumerate(b):
                out[i + j] = (out[i + j] + x * y) % R
    return out


def padd(a, b):
    n = max(len(a), len(b))
    return [((a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0)) % R for i in range(n)]


def gate_poly(gate, d, polys):
    if gate == 1:
        qL, qR, qM, qO, qC, a, b, c = polys
        f = padd(pmul(qL, a), pmul(qR, b))
        f = padd(f, pmul(pmul(qM, a), b))
        f = padd(f, pmul(qO, c))
        return padd(f, qC)
    f = polys[0]
    for p in polys[1:d]:
        f = pmul(f, p)
    if gate & 0xFF == 2:
        return padd(f, [(-x) % R for x in polys[d]])
    for p in polys[d:d + (gate >> 8)]:
        f = padd(f, p)
    return f


def divide_by_zh(f, N):
    """long division of f by x^N - 1: returns (quotient, remainder)"""
    f = list(f)
    if len(f) <= N:
        return [0], f
    q = [0] * (len(f) - N)
    for k in range(len(f) - 1, N - 1, -1):
        cf = f[k]
        if cf:
            q[k - N] = cf
            f[k] = 0
            f[k - N] = (f[k - N] + cf) % R
    return q, f[:N]


def ntt_domain(n, d, logb=None):
    """Points of the NTT domain and its header word.  logb: None (default
    2^ceil(log2 d) N), k (2^k N points), or (k, s): the step-radix domain
    {7 w_{2^k N}^i} u {7 w_{2^(k+1) N} w_{2^s N}^i}."""
    if logb is None:
        logb = (d - 1).bit_length()
    if isinstance(logb, tuple):
        k, s = logb
        Mb, Ms = 1 << (n + k), 1 << (n + s)
        sigma = 7 * omega(n + k + 1) % R
        pts = [7 * pow(omega(n + k), i, R) % R for i in range(Mb)]
        pts += [sigma * pow(omega(n + s), i, R) % R for i in range(Ms)]
        return pts, (n + k) | ((n + s + 1) << 8)
    M = 1 << (n + logb)
    return [7 * pow(omega(n + logb), i, R) % R for i in range(M)], n + logb


def interpolate(points, vals):
    """Lagrange: the coefficients of the degree < len(points) polynomial."""
    m = len(points)
    out = [0] * m
    for i, (xi, yi) in enumerate(zip(points, vals)):
        num, den = [1], 1
        for j, xj in enumerate(points):
            if j != i:
                num = pmul(num, [(-xj) % R, 1])
                den = den * (xi - xj) % R
        sc = yi * inv(den) % R
        for t, cf in enumerate(num):
            out[t] = (out[t] + cf * sc) % R
    return out


def prove_ntt(gate, n, d, cols_int, logb=None):
    N = 1 << n
    pts, word = ntt_domain(n, d, logb)
    M = len(pts)
    coefs = [interpolate_h(c) for c in cols_int]
    f = gate_poly(gate, d, coefs)
    q, rem = divide_by_zh(f, N)
    if all(x == 0 for x in rem):
        q = (q + [0] * M)[:M]
    else:
        # f does not vanish on H: q is the degree < M interpolant of f / z_H
        # on the domain's points
        vals = [horner(f, x) * inv(pow(x, N, R) - 1) % R for x in pts]
        q = interpolate(pts, vals)
    qroot = merkle_root(q)
    tr = Transcript(2, gate, n, d, word)
    for col in cols_int:
        tr.absorb(merkle_root(col))
    tr.absorb(qroot)
    while True:
        z = tr.squeeze()
        if pow(z, N, R) != 1:
            break
    out = b"ZCN1" + b"".join(x.to_bytes(4, "little") for x in (gate, n, d, word)) + qroot
    for cf in coefs:
        out += enc(horner(cf, z))
    out += enc(horner(q, z))
    return out, q, z


# ------------------------------------------------- hash-based PCS ---

def pcs_rows(col, nc):
    w = 1 << nc
    return [col[i:i + w] for i in range(0, len(col), w)]


def rs_encode(row, logW):
    """Values of the polynomial with coefficients `row` at 7 w_W^k, k < W (Horner)."""
    W = 1 << logW
    wW = omega(logW)
    return [horner(row, 7 * pow(wW, k, R) % R) for k in range(W)]


def pcs_tree(cols_int, nc):
    """Leaves (per codeword position: SHA of the per-column digests) and root."""
    logW = nc + 2
    E_all = [[rs_encode(r, logW) for r in pcs_rows(col, nc)] for col in cols_int]
    W = 1 << logW
    leaves = []
    for k in range(W):
        dg = b"".join(sha(b"".join(enc(E[i][k]) for i in range(len(E)))) for E in E_all)
        leaves.append(sha(dg))
    levels = [leaves]
    while len(levels[-1]) > 1:
        lv = levels[-1]
        levels.append([sha(lv[2 * u] + lv[2 * u + 1]) for u in range(len(lv) // 2)])
    return E_all, levels, sha(W.to_bytes(8, "little") + levels[-1][0])


def eq_tab(x):
    k = len(x)
    return [eq(x, bits_msb(b, k)) if k else 1 for b in range(1 << k)]


def pcs_open(n, nc, cols_int, alpha, values, t):
    """The PCS opening restated: u_j with eq over alpha_1..nr, gamma, u' with
    gamma^(j m + i), t queried columns with their sibling paths."""
    E_all, levels, root = pcs_tree(cols_int, nc)
    nr = n - nc
    m, w, W = 1 << nr, 1 << nc, 1 << (nc + 2)
    st = sha(b"zerocheck-gb300/pcs-v1" + b"".join(x.to_bytes(4, "little") for x in (n, nc, len(cols_int), t))
             + root + b"".join(enc(a) for a in alpha) + b"".join(enc(v) for v in values))
    tr = Transcript.__new__(Transcript)
    tr.s = st
    eh = eq_tab(alpha[:nr])
    rows = [pcs_rows(col, nc) for col in cols_int]
    us = [[sum(eh[i] * rows[j][i][l] for i in range(m)) % R for l in range(w)] for j in range(len(cols_int))]
    ub = b"".join(enc(x) for u in us for x in u)
    tr.absorb(ub)
    g = tr.squeeze()
    up = [sum(pow(g, j * m + i, R) * rows[j][i][l] for j in range(len(cols_int)) for i in range(m)) % R
          for l in range(w)]
    upb = b"".join(enc(x) for x in up)
    tr.absorb(upb)
    out = b"ZCP1" + b"".join(x.to_bytes(4, "little") for x in (n, nc, len(cols_int), t)) + ub + upb
    for _ in range(t):
        k = tr.squeeze() & (W - 1)
        out += b"".join(enc(enc_row[k]) for E in E_all for enc_row in E)
        idx = k
        for lv in levels[:-1]:
            out += lv[idx ^ 1]
            idx >>= 1
    return out, root, us
