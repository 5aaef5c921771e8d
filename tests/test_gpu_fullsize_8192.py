"""The 8192 workload at full size through the C ABI against the oracle:
m = n = k = 8192, BF16 operands with sigma_i = (1+i/16)^-2, r = 512, p = 32,
q = 1 (l = 544: the two-level Cholesky and the widest small SVD).

* The bench's recipe: INT8 E1 and E2, E3 split into a lead of the 64
  largest rank directions in INT8 with both split-precision residual terms
  and an MXFP4 tail (32-element blocks), tensor-core range finder (BF16
  operands exact on kind::f16) and TF32 factor assembly -- against the
  oracle's lead / tail chain on the oracle's FP64 factors by the
  quantisation-noise criterion of the other quantised end-to-end tests.
* The FP32 path (no quantisation, FP32 products): <= 1e-5.
Both on a seeded sample of 256 output rows, which the oracle forms exactly
(per-row scales and 32-element blocks along K make each output row depend
on that row of U~ alone).
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


@pytest.fixture(scope="module")
def w8192():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    A, B = workloads.device_operands("lramm_8192", torch.device("cuda", 0))
    c = workloads.CONFIGS["lramm_8192"]
    Ah, Bh = A.float().cpu().numpy(), B.float().cpu().numpy()   # BF16 widens exactly
    fac = oracle.lramm.factors(Ah, Bh, c["r"], c["p"], c["q"], workloads.SEED_SKETCH)
    rows = np.sort(np.random.default_rng(5).choice(c["m"], 256, replace=False))
    exact = oracle.lramm.exact_product(Ah[rows], Bh)
    return A, B, fac, rows, exact


def _run(L, A, B, rows, **kw):
    c = workloads.CONFIGS["lramm_8192"]
    plan = L.Plan(c["m"], c["n"], c["k"], c["r"], c["p"], c["q"], seed=workloads.SEED_SKETCH, a_type=L.BF16,
                  b_type=L.BF16, **kw)
    ws = plan.workspace()
    D = L.matmul(plan, A, B, ws=ws)
    info = L.info_read(ws, 4)
    assert L.status_read(ws) == 0
    out = D[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    del D, ws
    torch.cuda.empty_cache()
    return out, info


def test_lramm_8192_lead_tail_bench_configuration(L, w8192):
    A, B, (Ut, V, W, Zt), rows, exact = w8192
    D, info = _run(L, A, B, rows, prec=(1, 1, 4), lead=64, lead_prec=1, lead_split=2, sketch=L.SKETCH_TF32)
    assert int(info[3]) & 1   # factors assembled on the TF32 tensor cores
    ref_q = MX.chain_lead_tail(Ut[rows], V, W, Zt, (1, 1, 4), 64, 1, 2)
    ref_f = oracle.lramm.chain(Ut[rows], V, W, Zt, (0, 0, 0))
    quantised_agreement(D, ref_q, ref_f, exact)


def test_lramm_8192_fp32_path(L, w8192):
    A, B, (Ut, V, W, Zt), rows, _ = w8192
    D, _ = _run(L, A, B, rows, prec=(0, 0, 0), sketch=L.SKETCH_F32)
    ref = oracle.lramm.chain(Ut[rows], V, W, Zt, (0, 0, 0))
    assert oracle.lramm.rel_fro(D, ref) <= 1e-5
