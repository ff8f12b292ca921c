"""The step's two proofs run concurrently, as the benchmark runs them: the
SumCheck form (Sec. 3.3) on one context and stream, the NTT form (Sec. 3.2)
on another, forked from one event and joined back, several steps in a row
with nothing waiting on the device in between.  Every proof and quotient
must equal the oracle's byte for byte, as when each runs alone; sizes where
the SumCheck form uses its cooperative round kernel (n >= 14) beside the
NTT passes, and the host-thread variant of the end-to-end line."""
import concurrent.futures as cf

import numpy as np
import pytest

import oracle
from gpu_util import proof_bytes, to_device
from paper_2606_16146_gb300 import witness, zc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctxs():
    a = zc.Context(0, max_n=20, max_d=8)
    b = zc.Context(0, max_n=20, max_d=8)
    yield a, b
    a.close()
    b.close()


@pytest.mark.parametrize("gate,n,d,seed", [(1, 12, 3, 31), (1, 16, 3, 32), (1, 18, 3, 33), (2, 16, 4, 34),
                                           (1, 17, 3, 35)])
def test_two_streams_joined_every_step(ctxs, gate, n, d, seed):
    import torch
    ctx_nt, ctx_sc = ctxs
    tamper = seed == 35  # a witness that does not satisfy the gate, too
    cols = witness.generate(gate, n, d, seed, tamper=tamper)
    want_sc = oracle.prove_sumcheck(gate, n, d, cols)
    want_p, want_q = oracle.prove_ntt(gate, n, d, cols)
    dcols = to_device(cols)
    roots = [oracle.root(c) for c in cols]
    s_nt, s_sc = torch.cuda.Stream(), torch.cuda.Stream()
    steps = 3
    p_sc = [torch.zeros(zc.proof_size(gate, n, d, 1), dtype=torch.uint8, device="cuda") for _ in range(steps)]
    p_nt = [torch.zeros(zc.proof_size(gate, n, d, 2), dtype=torch.uint8, device="cuda") for _ in range(steps)]
    q = [torch.zeros(len(want_q), dtype=torch.uint8, device="cuda") for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        fork = torch.cuda.Event()
        fork.record(s_nt)
        s_sc.wait_event(fork)
        ctx_sc.prove_sumcheck(gate, n, d, dcols, roots=roots, stream=s_sc, proof_out=p_sc[k])
        ctx_nt.prove_ntt(gate, n, d, dcols, roots=roots, stream=s_nt, proof_out=p_nt[k], q_out=q[k])
        join = torch.cuda.Event()
        join.record(s_sc)
        s_nt.wait_event(join)
    torch.cuda.synchronize()
    for k in range(steps):
        assert proof_bytes(p_sc[k]) == want_sc
        assert proof_bytes(p_nt[k]) == want_p
        assert q[k].cpu().numpy().tobytes() == want_q.tobytes()


def test_two_host_threads_two_contexts(ctxs):
    """The end-to-end variant: the two calls from two host threads, host
    columns and host outputs."""
    ctx_nt, ctx_sc = ctxs
    gate, n, d = 1, 15, 3
    cols = witness.generate(gate, n, d, 36)
    want_sc = oracle.prove_sumcheck(gate, n, d, cols)
    want_p, want_q = oracle.prove_ntt(gate, n, d, cols)
    roots = [oracle.root(c) for c in cols]
    with cf.ThreadPoolExecutor(2) as ex:
        for _ in range(3):
            f_nt = ex.submit(ctx_nt.prove_ntt, gate, n, d, cols, roots=roots)
            f_sc = ex.submit(ctx_sc.prove_sumcheck, gate, n, d, cols, roots=roots)
            p, qq = f_nt.result()
            assert proof_bytes(f_sc.result()) == want_sc
            assert proof_bytes(p) == want_p
            assert np.asarray(qq).tobytes() == want_q.tobytes()
