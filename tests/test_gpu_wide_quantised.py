"""Quantised chains with l = r + p between 320 and 544, through lramm_matmul.

Inside lramm_matmul a quantised chain takes the small SVD in its M-only
form: the Jacobi rotates M = R^T alone and the right factors are formed as
P1 (R1 U_s Sigma^-1) from the first CholeskyQR pass of the projection.
Above l = 320 that form runs shapes the V-accumulating pair kernel does not
(blocks of 11 to 17 columns).  Two chains, both on the loose Jacobi
stopping rule of quantised chains: the plain INT8 chain at l = 400, and the
lead / tail chain of the 8192 workload's recipe (INT8 E1 and E2, INT8 lead
with both residual terms, MXFP4 tail) at l = 544.  Each is compared with the oracle's
quantised chain on the oracle's FP64 factors by the noise criterion of the
other quantised end-to-end tests.  Each runs with FP32 range-finder
products and with TF32 tensor-core ones; in the TF32 mode the factors of
these chains are assembled by TF32 tensor-core products too (the library
reports it in info word 3), the path the 8192 workload's bench figure uses.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests.test_gpu_parity import quantised_agreement

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
MX = oracle.mixed


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_16917_gb300 as L
    L.load()
    return L


def _run(L, plan, A32, B32, sketch):
    ws = plan.workspace()
    D = L.matmul(plan, torch.from_numpy(A32).cuda(), torch.from_numpy(B32).cuda(), ws=ws)
    info = L.info_read(ws, 4)
    assert L.status_read(ws) == 0
    # info word 3, bit 0: the factors were assembled on the TF32 tensor cores
    assert (int(info[3]) & 1) == (1 if sketch == L.SKETCH_TF32 else 0)
    return D.cpu().numpy().astype(np.float64)


SKETCHES = ["f32", "tf32"]


def _mode(L, name):
    return L.SKETCH_TF32 if name == "tf32" else L.SKETCH_F32


@pytest.mark.parametrize("sketch", SKETCHES)
def test_int8_chain_l400(L, sketch):
    m, n, k, r, p, q = 600, 560, 640, 380, 20, 1
    A, B = workloads.operands("lramm_4096", scale=(m, n, k))
    A32, B32 = A.astype(np.float32), B.astype(np.float32)
    sk = _mode(L, sketch)
    D = _run(L, L.Plan(m, n, k, r, p, q, seed=7, prec=(1, 1, 1), sketch=sk), A32, B32, sk)
    fac = oracle.lramm.factors(A32, B32, r, p, q, 7)
    ref_q = oracle.lramm.chain(*fac, (1, 1, 1))
    ref_f = oracle.lramm.chain(*fac, (0, 0, 0))
    quantised_agreement(D, ref_q, ref_f, oracle.lramm.exact_product(A32, B32))


@pytest.mark.parametrize("sketch", SKETCHES)
def test_lead_tail_chain_l544(L, sketch):
    m = n = k = 600
    r, p, q, lead = 512, 32, 1, 64
    A, B = workloads.operands("lramm_8192", scale=(m, n, k))
    A32, B32 = A.astype(np.float32), B.astype(np.float32)
    sk = _mode(L, sketch)
    plan = L.Plan(m, n, k, r, p, q, seed=7, prec=(1, 1, 4), lead=lead, lead_prec=1, lead_split=2, sketch=sk)
    D = _run(L, plan, A32, B32, sk)
    fac = oracle.lramm.factors(A32, B32, r, p, q, 7)
    ref_q = MX.chain_lead_tail(*fac, (1, 1, 4), lead, 1, 2)
    ref_f = oracle.lramm.chain(*fac, (0, 0, 0))
    quantised_agreement(D, ref_q, ref_f, oracle.lramm.exact_product(A32, B32))
