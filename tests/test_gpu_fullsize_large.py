"""The two large workloads at full size through the C ABI against the oracle.

lramm_32768 (m = n = 32768, k = 4096, sigma_i = (1+i)^-1.5, r = 128, p = 16,
q = 2, INT8 factors): the oracle's randomized SVDs run in full (FP64); the
m x n output is compared on a seeded sample of 256 rows, which the oracle
computes exactly (with per-row scales on the left factor and per-column
scales on E2, a row of D depends only on that row of U~).  Its "forward and
backward" runs the same operands through the range-finder form (forward on
the sampled rows, both gradients in full).

rf_linear (X 16384 x 4096 BF16, W 4096 x 11008 FP32, sigma_i =
exp(-i/128) + 1e-3, r = 384, p = 16, q = 1): forward in FP32 and with FP8
(e4m3) factors, and the hand-written backward, against the oracle in full.
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


# ------------------------------------------------------------- lramm_32768
@pytest.fixture(scope="module")
def big():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    A, B = workloads.device_operands("lramm_32768", torch.device("cuda", 0))
    c = workloads.CONFIGS["lramm_32768"]
    Ah, Bh = A.cpu().numpy(), B.cpu().numpy()
    fac = oracle.lramm.factors(Ah, Bh, c["r"], c["p"], c["q"], workloads.SEED_SKETCH)
    rows = np.sort(np.random.default_rng(5).choice(c["m"], 256, replace=False))
    exact = oracle.lramm.exact_product(Ah[rows], Bh)
    return A, B, fac, rows, exact


def _run_big(L, A, B, prec, sketch, rows):
    c = workloads.CONFIGS["lramm_32768"]
    plan = L.Plan(c["m"], c["n"], c["k"], c["r"], c["p"], c["q"], seed=workloads.SEED_SKETCH, prec=prec,
                  sketch=sketch)
    ws = plan.workspace()
    D = L.matmul(plan, A, B, ws=ws)
    assert L.status_read(ws) == 0
    out = D[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    del D, ws
    torch.cuda.empty_cache()
    return out


def test_lramm_32768_fp32_path(L, big):
    A, B, (Ut, V, W, Zt), rows, _ = big
    D = _run_big(L, A, B, (0, 0, 0), L.SKETCH_F32, rows)
    ref = oracle.lramm.chain(Ut[rows], V, W, Zt, (0, 0, 0))
    assert oracle.lramm.rel_fro(D, ref) <= 1e-5


def test_lramm_32768_int8_bench_configuration(L, big):
    A, B, (Ut, V, W, Zt), rows, exact = big
    D = _run_big(L, A, B, (1, 1, 1), L.SKETCH_TF32, rows)
    ref_q = oracle.lramm.chain(Ut[rows], V, W, Zt, (1, 1, 1))
    ref_f = oracle.lramm.chain(Ut[rows], V, W, Zt, (0, 0, 0))
    quantised_agreement(D, ref_q, ref_f, exact)


# ------------------------------------------------------------- rf_linear
@pytest.fixture(scope="module")
def rf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda", 0)
    X32, W = workloads.device_operands("rf_linear", dev, dtype=torch.float32)
    X = X32.to(torch.bfloat16)
    c = workloads.CONFIGS["rf_linear"]
    g = torch.Generator(device=dev)
    g.manual_seed(17)
    G = torch.randn((c["m"], c["n"]), generator=g, device=dev, dtype=torch.float32)
    return X, W, G, X.float().cpu().numpy(), W.cpu().numpy()


def _rf_plan(L, prec, sketch):
    c = workloads.CONFIGS["rf_linear"]
    return L.Plan(c["m"], c["n"], c["k"], c["r"], c["p"], c["q"], seed=workloads.SEED_SKETCH, prec=(0, 0, prec),
                  sketch=sketch, a_type=L.BF16, b_type=L.F32)


def test_rf_linear_forward_fp32(L, rf):
    X, W, _, Xh, Wh = rf
    c = workloads.CONFIGS["rf_linear"]
    plan = _rf_plan(L, 0, L.SKETCH_F32)
    ws = plan.workspace()
    C = L.rf_forward(plan, X, W, ws=ws).cpu().numpy().astype(np.float64)
    assert L.status_read(ws) == 0
    ref = oracle.rf.rf_forward(Xh, Wh, c["r"], c["p"], c["q"], workloads.SEED_SKETCH)
    assert oracle.lramm.rel_fro(C, ref) <= 1e-5


def test_rf_linear_forward_e4m3_bench_configuration(L, rf):
    X, W, _, Xh, Wh = rf
    c = workloads.CONFIGS["rf_linear"]
    plan = _rf_plan(L, 3, L.SKETCH_TF32)
    ws = plan.workspace()
    C = L.rf_forward(plan, X, W, ws=ws).cpu().numpy().astype(np.float64)
    assert L.status_read(ws) == 0
    ref_q = oracle.rf.rf_forward(Xh, Wh, c["r"], c["p"], c["q"], workloads.SEED_SKETCH, prec=3)
    ref_f = oracle.rf.rf_forward(Xh, Wh, c["r"], c["p"], c["q"], workloads.SEED_SKETCH)
    quantised_agreement(C, ref_q, ref_f, oracle.lramm.exact_product(Xh, Wh))


def test_rf_linear_backward(L, rf):
    X, W, G, Xh, Wh = rf
    c = workloads.CONFIGS["rf_linear"]
    plan = _rf_plan(L, 0, L.SKETCH_F32)
    ws = plan.workspace()
    dX, dW = (t.cpu().numpy().astype(np.float64) for t in L.rf_backward(plan, X, W, G, ws=ws))
    assert L.status_read(ws) == 0
    rX, rW = oracle.rf.rf_backward(Xh, Wh, G.cpu().numpy(), c["r"], c["p"], c["q"], workloads.SEED_SKETCH)
    assert oracle.lramm.rel_fro(dX, rX) <= 1e-4
    assert oracle.lramm.rel_fro(dW, rW) <= 1e-4


def test_lramm_32768_range_finder_forward_backward(L, big):
    """The 32768 workload's "forward and backward": its operands through the
    range-finder form C = (A Q)(Q^T B) (the differentiable form; the SVD form
    has no backward), FP32 path.  Forward on the 256 sampled rows <= 1e-5;
    the hand-written backward (dX = G P Q^T, dW through the QR adjoints of
    the q = 2 power chain) for a dense Gaussian G against the oracle's
    gradients, relative Frobenius <= 1e-4 over the full 32768 x 4096 and
    4096 x 32768 gradients."""
    A, B, _, rows, _ = big
    c = workloads.CONFIGS["lramm_32768"]
    plan = L.Plan(c["m"], c["n"], c["k"], c["r"], c["p"], c["q"], seed=workloads.SEED_SKETCH, prec=(0, 0, 0),
                  sketch=L.SKETCH_F32)
    ws = plan.workspace()
    C = L.rf_forward(plan, A, B, ws=ws)
    assert L.status_read(ws) == 0
    Cs = C[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    del C
    torch.cuda.empty_cache()
    g = torch.Generator(device=A.device)
    g.manual_seed(23)
    G = torch.randn((c["m"], c["n"]), generator=g, device=A.device, dtype=torch.float32)
    dX, dW = L.rf_backward(plan, A, B, G, ws=ws)
    assert L.status_read(ws) == 0
    dX, dW = dX.cpu().numpy().astype(np.float64), dW.cpu().numpy().astype(np.float64)
    Gh = G.cpu().numpy()
    del G, ws
    torch.cuda.empty_cache()
    Ah, Bh = A.cpu().numpy(), B.cpu().numpy()
    T, P, _ = oracle.rf.rf_factors(Ah, Bh, c["r"], c["p"], c["q"], workloads.SEED_SKETCH)
    assert oracle.lramm.rel_fro(Cs, T[rows] @ P) <= 1e-5
    del T, P
    rX, rW = oracle.rf.rf_backward(Ah, Bh, Gh, c["r"], c["p"], c["q"], workloads.SEED_SKETCH)
    assert oracle.lramm.rel_fro(dX, rX) <= 1e-4
    assert oracle.lramm.rel_fro(dW, rW) <= 1e-4
