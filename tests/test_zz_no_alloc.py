"""zc_prove_sumcheck_static, the SumCheck prover for callers that cannot
allocate device memory while proving (fixed pools, allocation-free
pipelines): its proofs equal those of zc_prove_sumcheck, on two calls in a
row that share the library's static scratch.  Collected last on purpose."""
import pytest

from gpu_util import proof_bytes, to_device
from paper_2606_16146_gb300 import witness, zc

pytestmark = pytest.mark.gpu

CASES = [(1, 12, 3, 7), (2, 10, 5, 8), (1, 16, 3, 9)]


def test_static_scratch_matches_context_prover():
    import torch
    ctx = zc.Context(0, max_n=16, max_d=8)
    try:
        for gate, n, d, seed in CASES:
            cols = witness.generate(gate, n, d, seed)
            dcols = to_device(cols)
            want = proof_bytes(ctx.prove_sumcheck(gate, n, d, dcols))
            size = zc.proof_size(gate, n, d, zc.ZC_FORM_SUMCHECK)
            for call in range(2):              # the second call reuses the static arrays
                out = torch.zeros(size, dtype=torch.uint8, device="cuda")
                roots = None if call == 0 else ctx.roots(gate, n, d, dcols)
                zc.prove_sumcheck_static(gate, n, d, dcols, out, roots=roots)
                torch.cuda.synchronize()
                assert proof_bytes(out) == want, (gate, n, d, call)
    finally:
        ctx.close()


def test_static_scratch_rejects_oversized_instances():
    import torch
    gate, n, d = 1, 18, 3                      # 8 columns x 2^18 x 32 B = 64 MiB > 32 MiB
    cols = [torch.zeros(32 << n, dtype=torch.uint8, device="cuda") for _ in range(8)]
    out = torch.zeros(zc.proof_size(gate, n, d, zc.ZC_FORM_SUMCHECK), dtype=torch.uint8, device="cuda")
    with pytest.raises(zc.ZCError) as e:
        zc.prove_sumcheck_static(gate, n, d, cols, out)
    assert e.value.status == 5
