"""Write the oracle's outputs for the large workload sizes as digests.

The GPU parity tests at the configuration sizes (n = 22 and 24) compare the
library's proof and quotient bytes with these records, so the box does not
have to rerun the oracle for minutes per case.  Every record is produced
here by the CPU oracle (``oracle/``) on the seeded witness of
``paper_2606_16146_gb300.witness``; nothing else is called.

Record format (one JSON object per line of ``oracle_digests.jsonl``):
  form (1 SumCheck, 2 NTT, 3 eq-factored SumCheck, 5 commitment), gate, n,
  d, log_blowup (NTT; 0 = default; the query count for form 5), seed,
  proof_len, proof_sha256, q_len, q_sha256 (NTT only), root (form 5).

Usage (repository root):
  python tests/golden/make_oracle_digests.py            # every missing case
  python tests/golden/make_oracle_digests.py --all      # recompute everything
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2606_16146_gb300 import witness  # noqa: E402

OUT = os.path.join(HERE, "oracle_digests.jsonl")

# (form, gate, n, d, log_blowup, seed): the configuration sizes whose oracle
# run is too long for the GPU test session.  form 1 SumCheck, 2 NTT, 3 the
# eq-factored SumCheck.
#   configs: Plonk n = 20, 22 (seed 1000 + n); product gate n = 22,
#   d in {2, 4, 8, 16, 32} (seed 2000 + d), both forms; the served mix's
#   largest shapes at n = 24 (seed 6000 + d); Plonk n = 22 on the
#   quotient-sized 2N domain.
#   the sweep's other n = 22 rows: product d = 6 on 8N and 5N = 4N + N,
#   Plonk and product d = 4 on 3N = 2N + N, the eq-factored Plonk proof;
#   the family at n = 22 (sum gate, seed 7000 + 100 m + 10 d + n):
#   g1g2g3g4 and g1g2+g3+g4+g5, both forms;
#   form 5: the hash-based commitment of the bench's Plonk n = 22 columns
#   (root, and the opening at PCS_ALPHA to PCS_VALUES with t queries; t sits
#   in the log_blowup slot).
_FAMILY = [((3 << 8) | 3, 2, 7000 + 300 + 20 + 22), (3, 4, 7000 + 40 + 22)]
CASES = (
    [(1, 1, 22, 3, 0, 1022), (2, 1, 22, 3, 0, 1022), (2, 1, 22, 3, 1, 1022)]
    + [(form, 2, 22, d, 0, 2000 + d) for d in (2, 4, 8, 16, 32) for form in (1, 2)]
    + [(1, 2, 24, 8, 0, 6008), (1, 2, 24, 16, 0, 6016), (1, 1, 24, 3, 0, 6003), (2, 1, 24, 3, 0, 6003)]
    + [(3, 1, 22, 3, 0, 1022), (2, 1, 22, 3, 257, 1022), (2, 2, 22, 4, 257, 2004),
       (1, 2, 22, 6, 0, 2006), (2, 2, 22, 6, 0, 2006), (2, 2, 22, 6, 258, 2006)]
    + [(form, g, 22, d, 0, seed) for g, d, seed in _FAMILY for form in (1, 2)]
    + [(5, 1, 22, 3, 189, 1022)]
)


def pcs_point(n: int, c: int):
    """The opening point and claimed values of the commitment records: small
    integers (any values give well-defined opening bytes)."""
    alpha = [oracle.ints_to_bytes([x]).tobytes() for x in range(3, 3 + n)]
    values = [oracle.ints_to_bytes([7 + j]).tobytes() for j in range(c)]
    return alpha, values
# cheapest first, so an interrupted run still leaves the most records
CASES = sorted(CASES, key=lambda c: (1 << c[2]) * (c[3] + 2) * (1 if c[0] == 1 else 8 * max(c[3], 4)))


def key(rec) -> tuple:
    return (rec["form"], rec["gate"], rec["n"], rec["d"], rec["log_blowup"], rec["seed"])


def load(path: str = OUT) -> dict:
    recs = {}
    if os.path.exists(path):
        with open(path) as f:
            for line in f:
                line = line.strip()
                if line:
                    r = json.loads(line)
                    recs[key(r)] = r
    return recs


def compute(form, gate, n, d, lb, seed) -> dict:
    cols = witness.generate(gate, n, d, seed)
    rec = {"form": form, "gate": gate, "n": n, "d": d, "log_blowup": lb, "seed": seed}
    if form == 5:
        root = oracle.pcs_commit(n, cols)
        alpha, values = pcs_point(n, len(cols))
        proof = oracle.pcs_open(n, cols, alpha, values, lb)
        rec.update(root=root.hex(), proof_len=len(proof), proof_sha256=hashlib.sha256(proof).hexdigest())
    elif form in (1, 3):
        proof = (oracle.prove_sumcheck if form == 1 else oracle.prove_sumcheck_eq)(gate, n, d, cols)
        rec.update(proof_len=len(proof), proof_sha256=hashlib.sha256(proof).hexdigest())
    else:
        proof, q = oracle.prove_ntt(gate, n, d, cols, log_blowup=lb)
        qb = q.tobytes()
        rec.update(proof_len=len(proof), proof_sha256=hashlib.sha256(proof).hexdigest(),
                   q_len=len(qb), q_sha256=hashlib.sha256(qb).hexdigest())
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--all", action="store_true", help="recompute every case")
    args = ap.parse_args()
    recs = {} if args.all else load()
    for case in CASES:
        if case in recs:
            continue
        t0 = time.time()
        rec = compute(*case)
        recs[case] = rec
        with open(OUT + ".tmp", "w") as f:
            for c in CASES:
                if c in recs:
                    f.write(json.dumps(recs[c], sort_keys=True) + "\n")
        os.replace(OUT + ".tmp", OUT)
        print(f"{case}: {time.time() - t0:.1f} s", flush=True)


if __name__ == "__main__":
    main()
