"""The full lramm_4096 workload (m = n = k = 4096, r = 256, p = 16, q = 2,
sigma_i = (1+i)^-1) through the C ABI against the oracle at full size.

* FP32 path (FP32 sketch, FP32 factors): <= 1e-5 relative Frobenius.
* The launch configuration bench.py times (TF32 tensor-core sketch, INT8
  factors with per-row/column scales): the same quantisation-noise criterion
  as the small end-to-end tests -- the GPU's and the oracle's factors differ
  by rounding, so their quantised outputs are two draws of the same
  quantisation noise; both errors against the exact product agree to 10%.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests.test_gpu_parity import quantised_agreement

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_16917_gb300 as L
    L.load()
    return L


@pytest.fixture(scope="module")
def operands():
    A, B = workloads.operands("lramm_4096")
    return A.astype(np.float32), B.astype(np.float32)


def _run(L, A, B, prec, sketch):
    c = workloads.CONFIGS["lramm_4096"]
    m, k = A.shape
    n = B.shape[1]
    plan = L.Plan(m, n, k, c["r"], c["p"], c["q"], seed=workloads.SEED_SKETCH, prec=prec, sketch=sketch)
    ws = plan.workspace()
    D = L.matmul(plan, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), ws=ws)
    assert L.status_read(ws) == 0
    return D.cpu().numpy().astype(np.float64)


def test_fp32_path_full_size(L, operands):
    A, B = operands
    c = workloads.CONFIGS["lramm_4096"]
    D = _run(L, A, B, (0, 0, 0), L.SKETCH_F32)
    ref = oracle.lramm.lramm(A, B, c["r"], c["p"], c["q"], workloads.SEED_SKETCH, (0, 0, 0))
    assert oracle.lramm.rel_fro(D, ref) <= 1e-5


def test_int8_bench_configuration_full_size(L, operands):
    A, B = operands
    c = workloads.CONFIGS["lramm_4096"]
    D = _run(L, A, B, (1, 1, 1), L.SKETCH_TF32)
    ref_q = oracle.lramm.lramm(A, B, c["r"], c["p"], c["q"], workloads.SEED_SKETCH, (1, 1, 1))
    ref_f = oracle.lramm.lramm(A, B, c["r"], c["p"], c["q"], workloads.SEED_SKETCH, (0, 0, 0))
    quantised_agreement(D, ref_q, ref_f, oracle.lramm.exact_product(A, B))
