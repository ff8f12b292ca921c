"""Algorithmic work of one proof: modular multiplications and DRAM bytes.

These are the counts the roofline is taken against (per proof, by form):

SumCheck, per round pair and summed over all rounds (N - 1 pairs): the
eq-weighted gate at d + 1 points with g + 1 multiplications each
(g = 5 for the Plonk gate, d - 1 for the product and sum gates), the eq weight, and
one fold multiplication per column.  Bytes: every column read twice and
written once over the rounds (2 c N reads + c N writes, at 32 bytes, taken
as 128 c N bytes with the round-1 conversions).

NTT: c inverse NTTs of size N (N/2 log N butterflies each), c s forward
NTTs of size N on the coset slices plus their coset scaling, the gate at M
points, the quotient inverse NTT of size M, its scaling, and the openings
(c N + (d - 1) N).  Bytes: columns in, coefficients out and back in, one
slice pass per column and slice, q-hat out and in, q out, q read for the
root and the opening.  A step-radix domain of Mb + N points (Mb = 2^k N)
has s = 2^k + 1 slices; its quotient transform is the Mb-point inverse NTT
with its scaling, the reduction of q_big (Mb multiplications), an N-point
coset NTT of the reduced q_big and an N-point inverse NTT with their
scalings, and the combination (2 N).
"""
from __future__ import annotations

import math


def ncols(gate: int, d: int) -> int:
    if gate == 1:
        return 8
    return d + 1 if gate == 2 else d + (gate >> 8)


def blowup(d: int) -> int:
    return 1 << max(0, (d - 1).bit_length())


def domain(n: int, d: int, log_blowup: int = 0) -> tuple[int, int]:
    """(Mb, Ms): the power-of-two part and the step-radix part (0 if none)
    of the NTT domain for a domain word (0: next_pow2(d) N)."""
    N = 1 << n
    k, sp1 = log_blowup & 0xFF, (log_blowup >> 8) & 0xFF
    if not sp1:
        return (1 << k if k else blowup(d)) * N, 0
    return N << k, N << (sp1 - 1)


def algorithmic_mulmods(form: str, n: int, d: int = 3, gate: int = 1, log_blowup: int = 0) -> float:
    N = 1 << n
    c = ncols(gate, d)
    g = 5 if gate == 1 else d - 1
    if form == "sumcheck":
        return (N - 1) * ((d + 1) * (g + 1) + 1 + c)
    Mb, Ms = domain(n, d, log_blowup)
    M = Mb + Ms
    s = M / N
    q_transform = (Mb / 2) * math.log2(Mb) + Mb
    if Ms:
        q_transform += Mb + 2 * ((Ms / 2) * math.log2(Ms) + Ms) + 2 * Ms
    return (c * (N / 2) * n + c * s * (N + (N / 2) * n) + M * (g + 1)
            + q_transform + c * N + (d - 1) * N)


def algorithmic_bytes(form: str, n: int, d: int = 3, gate: int = 1, log_blowup: int = 0) -> float:
    N = 1 << n
    c = ncols(gate, d)
    if form == "sumcheck":
        return 128.0 * c * N
    Mb, Ms = domain(n, d, log_blowup)
    M = Mb + Ms
    return 32.0 * (2 * c * N + c * M + M + 2 * M + c * N + M)
