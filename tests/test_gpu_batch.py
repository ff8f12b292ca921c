"""Batched proving: a mixed batch of SumCheck and NTT instances of different
sizes, gates and degrees proves, on concurrent lanes and as one captured
CUDA graph, exactly the bytes each instance proves alone (the arithmetic of
Fig. side-by-side-zc is per instance; batching only changes scheduling)."""
import numpy as np
import pytest

import oracle
from gpu_util import proof_bytes, to_device
from paper_2606_16146_gb300 import witness, zc

pytestmark = pytest.mark.gpu

# (form, gate, n, d)
MIX = [
    (1, 1, 10, 3), (2, 1, 9, 3), (1, 2, 7, 8), (2, 2, 6, 8), (1, 1, 1, 3),
    (2, 1, 12, 3), (1, 1, 13, 3), (2, 2, 3, 4), (1, 2, 11, 2), (2, 1, 2, 3),
    (1, 1, 5, 3), (2, 2, 10, 5), (1, 2, 4, 16), (2, 1, 14, 3),
]


@pytest.fixture(scope="module")
def ctx():
    c = zc.Context(0, max_n=24, max_d=32)
    yield c
    c.close()


def _expected(form, gate, n, d, cols):
    if form == 1:
        return oracle.prove_sumcheck(gate, n, d, cols), None
    p, q = oracle.prove_ntt(gate, n, d, cols)
    return p, q.tobytes()


def _setup(mix, seed0):
    import torch
    insts = []
    for i, (form, gate, n, d) in enumerate(mix):
        cols = witness.generate(gate, n, d, seed0 + i)
        size = zc.proof_size(gate, n, d, form)
        proof = torch.zeros(size, dtype=torch.uint8, device="cuda")
        q = None
        if form == 2:
            lb = 0
            while (1 << lb) < d:
                lb += 1
            q = torch.zeros(32 << (n + lb), dtype=torch.uint8, device="cuda")
        insts.append(dict(form=form, gate=gate, n=n, d=d, cols=cols, dcols=to_device(cols),
                          proof=proof, q=q))
    return insts


def _args(insts):
    return ([x["form"] for x in insts], [(x["gate"], x["n"], x["d"], 0) for x in insts],
            [x["dcols"] for x in insts], [x["proof"] for x in insts], [x["q"] for x in insts])


def _check_all(insts):
    for x in insts:
        want_p, want_q = _expected(x["form"], x["gate"], x["n"], x["d"], x["cols"])
        assert proof_bytes(x["proof"]) == want_p, (x["form"], x["gate"], x["n"], x["d"])
        if want_q is not None:
            assert x["q"].cpu().numpy().tobytes() == want_q


def test_prove_batch_matches_single(ctx):
    import torch
    insts = _setup(MIX, 7000)
    forms, params, cols, proofs, qs = _args(insts)
    ctx.prove_batch(forms, params, cols, proofs, qs)
    torch.cuda.synchronize()
    _check_all(insts)


def test_batch_single_instance_and_no_q(ctx):
    import torch
    insts = _setup([(2, 1, 11, 3)], 7100)
    forms, params, cols, proofs, _ = _args(insts)
    ctx.prove_batch(forms, params, cols, proofs, None)
    torch.cuda.synchronize()
    want_p, _ = _expected(2, 1, 11, 3, insts[0]["cols"])
    assert proof_bytes(insts[0]["proof"]) == want_p


def test_batch_graph_relaunch_reads_current_columns(ctx):
    import torch
    insts = _setup(MIX[:8], 7200)
    forms, params, cols, proofs, qs = _args(insts)
    g = ctx.batch_graph(forms, params, cols, proofs, qs)
    try:
        assert g.kernels > len(insts)
        g.launch()
        torch.cuda.synchronize()
        _check_all(insts)
        # new witnesses into the same buffers, zeroed outputs: a relaunch proves them
        for i, x in enumerate(insts):
            x["cols"] = witness.generate(x["gate"], x["n"], x["d"], 7300 + i)
            for dst, src in zip(x["dcols"], x["cols"]):
                dst.copy_(torch.from_numpy(np.ascontiguousarray(src)))
            x["proof"].zero_()
            if x["q"] is not None:
                x["q"].zero_()
        g.launch()
        g.launch()
        torch.cuda.synchronize()
        _check_all(insts)
    finally:
        g.close()


def test_batch_bad_arguments(ctx):
    insts = _setup([(1, 1, 4, 3)], 7400)
    forms, params, cols, proofs, qs = _args(insts)
    with pytest.raises(zc.ZCError):
        ctx.prove_batch([9], params, cols, proofs, qs)      # no such form
    with pytest.raises(zc.ZCError):
        ctx.prove_batch(forms, [(1, 30, 3, 0)], cols, proofs, qs)
