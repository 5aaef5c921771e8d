"""Failure detection on the GPU without a fault: a bounded wait that runs out.

The small SVD's thread-block cluster hands column blocks between CTAs with
bulk copies counted on mbarriers, every wait bounded.  With the test flags
one CTA skips its first block move and the waits give up after ~2^20 SM
cycles: the launch must latch LRAMM_ERR_TIMEOUT in the status word, return
(each CTA first waits, bounded, for the copies already issued into it), and
leave the context usable -- the same library calls then give the oracle's
result.  Both cluster kernels are covered: the one lramm_rsvd runs (V_s
accumulated) and the M-only one of quantised chains in lramm_matmul.
"""
import time

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_16917_gb300 as L
    L.load()
    return L


def test_rsvd_cluster_timeout_then_recovers(L):
    m, k, r, p, q = 600, 500, 60, 8, 1          # l = 68: a 5-CTA cluster
    X = workloads.lowrank(m, k, workloads.spectrum("exp32", min(m, k)), 91).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    bad = L.Plan(m, m, k, r, p, q, seed=7, test_flags=L.FLAG_SHORT_WAITS | L.FLAG_TEST_DROP_MOVE)
    ws = bad.workspace()
    t0 = time.time()
    L.rsvd(bad, 0, Xd, ws=ws)
    st = L.status_read(ws)
    assert st == 6, st                                  # LRAMM_ERR_TIMEOUT
    assert time.time() - t0 < 60.0
    good = L.Plan(m, m, k, r, p, q, seed=7)
    ws2 = good.workspace()
    U, S, V = (t.cpu().numpy() for t in L.rsvd(good, 0, Xd, ws=ws2))
    assert L.status_read(ws2) == 0
    Uo, so, Vo = oracle.lramm.rsvd(X, r, p, q, 7, 0)
    assert oracle.lramm.rel_fro((U * S) @ V.T, (Uo * so) @ Vo.T) < 1e-5


def test_matmul_monly_cluster_timeout_then_recovers(L):
    m = n = k = 512
    r, p, q = 64, 16, 1                                 # l = 80: the M-only kernel on a 5-CTA cluster
    A, B = workloads.operands("lramm_512", scale=(m, n, k))
    A32, B32 = A.astype(np.float32), B.astype(np.float32)
    Ad, Bd = torch.from_numpy(A32).cuda(), torch.from_numpy(B32).cuda()
    bad = L.Plan(m, n, k, r, p, q, seed=7, prec=(1, 1, 1),
                 test_flags=L.FLAG_SHORT_WAITS | L.FLAG_TEST_DROP_MOVE)
    ws = bad.workspace()
    L.matmul(bad, Ad, Bd, ws=ws)
    assert L.status_read(ws) == 6
    good = L.Plan(m, n, k, r, p, q, seed=7, prec=(1, 1, 1))
    ws2 = good.workspace()
    D = L.matmul(good, Ad, Bd, ws=ws2).cpu().numpy().astype(np.float64)
    assert L.status_read(ws2) == 0
    ref_q = oracle.lramm.lramm(A32, B32, r, p, q, 7, (1, 1, 1))
    ref_f = oracle.lramm.lramm(A32, B32, r, p, q, 7, (0, 0, 0))
    assert oracle.lramm.rel_fro(D, ref_q) <= 1.5 * oracle.lramm.rel_fro(ref_q, ref_f)


def test_flags_refused_outside_their_bits(L):
    with pytest.raises(L.LrammError) as e:
        L.Plan(64, 64, 64, 8, 4, 0, test_flags=16)
    assert e.value.code == 1
