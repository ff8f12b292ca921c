"""Seeded instance lists for the batched and served deployment modes.

Holds no prover arithmetic: only which shapes (gate, n, d), seeds and
arrival times a run uses.

* Batched: 64 instances; n drawn log-uniform over 2^10..2^20 rows (so n is
  uniform over the integers 10..20); degree 3 (Plonk gate) or 8 (product
  gate) with equal probability (sampler seed 3); instance i uses witness
  seed 3000 + i.
* Served: Poisson arrivals at a given rate; n uniform over 12..24; degree
  uniform over {3, 8, 16} (3: Plonk gate, otherwise the product gate);
  arrival/shape seed 4.  A request carries the seed of its shape's witness,
  so requests of one shape share device-resident columns (the witness pool):
  generating a fresh 0.5-9 GB witness per request on the host would take
  seconds per request and the loop would measure the generator.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import witness

PLONK, PRODUCT = witness.GATE_PLONK, witness.GATE_PRODUCT


@dataclass(frozen=True)
class Shape:
    gate: int
    n: int
    d: int

    @property
    def ncols(self) -> int:
        return witness.ncols(self.gate, self.d)


def gate_for_degree(d: int) -> int:
    return PLONK if d == 3 else PRODUCT


def batched_instances(count: int = 64, sampler_seed: int = 3, witness_seed0: int = 3000,
                      n_lo: int = 10, n_hi: int = 20):
    """[(Shape, witness_seed)] of the batched workload."""
    rng = np.random.default_rng(sampler_seed)
    out = []
    for i in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        d = 3 if rng.random() < 0.5 else 8
        out.append((Shape(gate_for_degree(d), n, d), witness_seed0 + i))
    return out


def shape_seed(s: Shape) -> int:
    """Witness seed of a shape in the served pool."""
    return 5000 + 100 * s.n + s.d


def served_requests(rate: float, count: int, seed: int = 4, n_lo: int = 12, n_hi: int = 24,
                    degrees=(3, 8, 16)):
    """[(arrival_s, Shape)] with exponential inter-arrival times of mean 1/rate.
    One seed gives the same shape sequence at every rate (arrivals scale by 1/rate)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for i in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        d = int(degrees[int(rng.integers(0, len(degrees)))])
        out.append((float(t[i]), Shape(gate_for_degree(d), n, d)))
    return out
