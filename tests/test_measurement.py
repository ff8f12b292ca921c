"""Host logic behind the bench line's roofline (no GPU): the algorithmic work
counts of both forms at sizes small enough to count by hand, the NTT domain
words, and the rule that a committed DRAM-traffic record is reported only
while the kernel sources still hash to the digest it was taken on."""
import hashlib
import importlib.util
import os

from paper_2606_16146_gb300 import costs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_sumcheck_counts_by_hand():
    # Plonk, n = 3: N - 1 = 7 pair-rounds, each (d + 1)(g + 1) = 4 * 6 gate
    # products, one eq weight and c = 8 folds
    assert costs.algorithmic_mulmods("sumcheck", 3, 3, 1) == 7 * (24 + 1 + 8)
    # product gate d = 4, n = 2: c = 5 columns, g = d - 1 = 3
    assert costs.algorithmic_mulmods("sumcheck", 2, 4, 2) == 3 * (5 * 4 + 1 + 5)
    # every column read twice and written once over the rounds, 32-byte
    # elements, with round 1's conversions: 128 c N bytes
    assert costs.algorithmic_bytes("sumcheck", 3, 3, 1) == 128 * 8 * 8


def test_ntt_counts_by_hand():
    # Plonk, n = 2: N = 4, M = 16 (s = 4 slices), c = 8, g = 5
    inverse = 8 * 2 * 2                 # c (N/2) n
    slices = 8 * 4 * (4 + 2 * 2)        # c s (N + (N/2) n): coset scaling and the slice NTTs
    gate = 16 * 6                       # M (g + 1)
    quotient = 8 * 4 + 16               # (M/2) log M + M
    openings = 8 * 4 + 2 * 4            # c N + (d - 1) N
    assert costs.algorithmic_mulmods("ntt", 2, 3, 1) == inverse + slices + gate + quotient + openings
    # columns in, coefficients out and back, one slice pass per column and
    # slice, q-hat out and in, q out, q read for root and opening
    N, M, c = 4, 16, 8
    assert costs.algorithmic_bytes("ntt", 2, 3, 1) == 32 * (2 * c * N + c * M + M + 2 * M + c * N + M)


def test_domain_words():
    N = 1 << 10
    assert costs.domain(10, 3) == (4 * N, 0)            # next_pow2(3) N
    assert costs.domain(10, 5) == (8 * N, 0)
    assert costs.domain(10, 3, 1) == (2 * N, 0)         # quotient-sized 2N
    assert costs.domain(10, 3, (1 << 8) | 1) == (2 * N, N)        # 3N = 2N + N
    assert costs.domain(10, 6, (1 << 8) | 2) == (4 * N, N)        # 5N = 4N + N
    # the step-radix domain costs less than the next power of two
    assert costs.algorithmic_mulmods("ntt", 20, 4, 2, (1 << 8) | 1) < costs.algorithmic_mulmods("ntt", 20, 4, 2)


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_record_follows_the_source_digest(tmp_path):
    bench = _bench()
    src = tmp_path / "kernel.cu"
    src.write_text("// a kernel\n")
    digest = hashlib.sha256(src.read_bytes()).hexdigest()
    rec = tmp_path / "record.md"
    rec.write_text("notes\n\ntraffic_bytes_per_launch: 2370000000\n"
                   f"sources: {src}\nsource_sha256: {digest}\n")
    assert bench.recorded_traffic(str(rec)) == 2370000000.0
    src.write_text("// the kernel changed\n")
    assert bench.recorded_traffic(str(rec)) is None
    rec.write_text("no record here\n")
    assert bench.recorded_traffic(str(rec)) is None

