"""zc_prove_sumcheck_static, the SumCheck prover for callers that cannot
allocate device memory while proving (fixed pools reserved up front,
stream-ordered pipelines that must not take the implicit synchronisation of
cudaMalloc/cudaFree): its proofs equal the oracle's and those of
zc_prove_sumcheck on calls in a row that share the library's static scratch,
the device's free memory does not move across calls, and instances beyond
the scratch are refused.  Collected last on purpose."""
import os

import pytest

import oracle
from gpu_util import proof_bytes, to_device
from paper_2606_16146_gb300 import witness, zc

pytestmark = pytest.mark.gpu

CASES = [(1, 12, 3, 7), (2, 10, 5, 8), (1, 16, 3, 9), (witness.gate_sum(1), 9, 2, 10)]


def test_static_scratch_matches_oracle_and_context_prover():
    import torch
    ctx = zc.Context(0, max_n=16, max_d=8)
    try:
        for gate, n, d, seed in CASES:
            cols = witness.generate(gate, n, d, seed)
            want = oracle.prove_sumcheck(gate, n, d, cols)
            dcols = to_device(cols)
            assert proof_bytes(ctx.prove_sumcheck(gate, n, d, dcols)) == want
            roots = ctx.roots(gate, n, d, dcols)
            size = zc.proof_size(gate, n, d, zc.ZC_FORM_SUMCHECK)
            outs = [torch.zeros(size, dtype=torch.uint8, device="cuda") for _ in range(3)]
            torch.cuda.synchronize()
            free = []
            for call in range(3):              # later calls reuse the static arrays
                zc.prove_sumcheck_static(gate, n, d, dcols, outs[call],
                                         roots=None if call != 1 else roots)
                torch.cuda.synchronize()
                free.append(torch.cuda.mem_get_info()[0])
                assert proof_bytes(outs[call]) == want, (gate, n, d, call)
            assert free[1] == free[2], "device memory changed across calls"
    finally:
        ctx.close()


def test_static_scratch_error_marker():
    """A column value >= r: the call returns at once and the proof starts with "ZCE!"."""
    import torch
    gate, n, d = 1, 6, 3
    cols = witness.generate(gate, n, d, 3)
    cols[2][32 * 5 + 31] = 0xff
    out = torch.zeros(zc.proof_size(gate, n, d, zc.ZC_FORM_SUMCHECK), dtype=torch.uint8, device="cuda")
    zc.prove_sumcheck_static(gate, n, d, to_device(cols), out)
    torch.cuda.synchronize()
    assert bytes(out[:4].cpu().numpy()) == b"ZCE!"


def test_static_scratch_rejects_oversized_instances():
    import torch
    gate, n, d = 1, 18, 3                      # 8 columns x 2^18 x 32 B = 64 MiB > 32 MiB
    cols = [torch.zeros(32 << n, dtype=torch.uint8, device="cuda") for _ in range(8)]
    out = torch.zeros(zc.proof_size(gate, n, d, zc.ZC_FORM_SUMCHECK), dtype=torch.uint8, device="cuda")
    with pytest.raises(zc.ZCError) as e:
        zc.prove_sumcheck_static(gate, n, d, cols, out)
    assert e.value.status == 5


def test_static_scratch_commitment_buffers_counted(monkeypatch):
    """An instance whose tables fit but whose commitment buffers (col_roots =
    NULL) do not is refused; the same instance with its roots given runs and
    gives the oracle's bytes.  The usable scratch is lowered to reach the
    boundary: the smallest limit that takes the instance with roots given."""
    import torch
    gate, n, d = 2, 11, 4
    cols = witness.generate(gate, n, d, 12)
    want = oracle.prove_sumcheck(gate, n, d, cols)
    roots = [oracle.root(c) for c in cols]
    dcols = to_device(cols)
    out = torch.zeros(zc.proof_size(gate, n, d, zc.ZC_FORM_SUMCHECK), dtype=torch.uint8, device="cuda")

    def fits(limit, with_roots):
        if limit is None:
            monkeypatch.delenv("ZC_STATIC_SCRATCH_BYTES", raising=False)
        else:
            monkeypatch.setenv("ZC_STATIC_SCRATCH_BYTES", str(limit))
        try:
            zc.prove_sumcheck_static(gate, n, d, dcols, out, roots=roots if with_roots else None)
        except zc.ZCError as e:
            assert e.status == 5
            return False
        torch.cuda.synchronize()
        return True

    lo, hi = 0, 32 << 20                        # smallest limit with roots given
    assert fits(hi, True)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if fits(mid, True):
            hi = mid
        else:
            lo = mid
    assert proof_bytes(out) == want
    assert not fits(hi, False), "commitment buffers not counted"
    assert fits(hi, True)
    assert proof_bytes(out) == want
    assert fits(None, False)                    # the full scratch takes it without roots
    assert proof_bytes(out) == want
    assert os.environ.get("ZC_STATIC_SCRATCH_BYTES") is None
