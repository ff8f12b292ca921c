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
root and the opening.
"""
from __future__ import annotations

import math


def ncols(gate: int, d: int) -> int:
    if gate == 1:
        return 8
    return d + 1 if gate == 2 else d + (gate >> 8)


def blowup(d: int) -> int:
    return 1 << max(0, (d - 1).bit_length())


def algorithmic_mulmods(form: str, n: int, d: int = 3, gate: int = 1, log_blowup: int = 0) -> float:
    N = 1 << n
    c = ncols(gate, d)
    g = 5 if gate == 1 else d - 1
    s = 1 << log_blowup if log_blowup else blowup(d)
    M = s * N
    if form == "sumcheck":
        return (N - 1) * ((d + 1) * (g + 1) + 1 + c)
    return (c * (N / 2) * n + c * s * (N + (N / 2) * n) + M * (g + 1)
            + (M / 2) * math.log2(M) + M + c * N + (d - 1) * N)


def algorithmic_bytes(form: str, n: int, d: int = 3, gate: int = 1, log_blowup: int = 0) -> float:
    N = 1 << n
    c = ncols(gate, d)
    M = (1 << log_blowup if log_blowup else blowup(d)) * N
    if form == "sumcheck":
        return 128.0 * c * N
    return 32.0 * (2 * c * N + c * M + M + 2 * M + c * N + M)
