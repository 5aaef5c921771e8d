"""The e4m3 range finder (LRAMM_SKETCH_E4M3) through the C ABI against the oracle.

Bars: the per-column quantiser bit-exact (codes and scales); the RSVD with
its range-finder products on e4m3 codes within 4 * 2^-10 (relative
Frobenius; singular values 2^-9) of the oracle's e4m3 RSVD on the same
input -- the two sides quantise the same FP32 operand and l-column matrices
whose values differ only by the FP32 orthonormalisation's rounding, so codes
rarely differ, and the projection B^T = X^T Q is a TF32 product on the GPU
(the bound of the TF32-sketch RSVD tests) against the oracle's exact one;
quantised end to end within the quantisation noise criterion of the other
end-to-end tests; at full size, the error of the approximation stays within
1% of the TF32 range finder's.
"""
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


def np_(t):
    return t.detach().cpu().numpy()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("prec", [1, 2, 3])
@pytest.mark.parametrize("rows,cols,ldc", [(4096, 272, 4096), (300, 37, 320), (1, 5, 32), (5000, 3, 5024)])
def test_quantize_cols_bit_exact(L, prec, rows, cols, ldc):
    rng = np.random.default_rng(rows + cols)
    X = (rng.standard_normal((rows, cols)) * np.exp(rng.uniform(-5, 5, (1, cols)))).astype(np.float32)
    X[:, min(2, cols - 1)] = 0.0
    codes, scales = L.quantize_cols(dev(X), prec, ldcodes=ldc)
    c = codes.float().cpu().numpy().astype(np.float64)
    oc, _, s = oracle.quant.quantize(X, prec, 0)
    assert np.array_equal(c[:, :rows], oc.T)
    assert np.all(c[:, rows:] == 0)
    assert np.array_equal(np_(scales), s)


@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("m,k,r,p,q", [(600, 500, 40, 8, 1), (1000, 700, 96, 16, 2), (333, 250, 20, 8, 0)])
def test_rsvd_e4m3_matches_oracle(L, which, m, k, r, p, q):
    X = workloads.lowrank(m, k, workloads.spectrum("poly1", min(m, k)), 800 + m).astype(np.float32)
    plan = (L.Plan(m, m, k, r, p, q, seed=7, sketch=L.SKETCH_E4M3) if which == 0
            else L.Plan(k, k, m, r, p, q, seed=7, sketch=L.SKETCH_E4M3))
    ws = plan.workspace()
    U, S, V = (np_(t).astype(np.float64) for t in L.rsvd(plan, which, dev(X), ws=ws))
    assert L.status_read(ws) == 0
    Uo, so, Vo = oracle.sketch8.rsvd_e4m3(X, r, p, q, 7, which)
    assert oracle.lramm.rel_fro((U * S) @ V.T, (Uo * so) @ Vo.T) < 4 * 2.0 ** -10
    assert np.allclose(S, so, rtol=2.0 ** -9, atol=2.0 ** -9 * so[0])
    # and the e4m3 range finder stays within 1% of the FP64 one's rank-r error
    U0, s0, V0 = oracle.lramm.rsvd(X, r, p, q, 7, which)
    e8 = np.linalg.norm(X - (U * S) @ V.T)
    assert e8 <= 1.01 * np.linalg.norm(X - (U0 * s0) @ V0.T)


def test_matmul_e4m3_sketch_quantised(L):
    """Algorithm 3 with the e4m3 range finder and the INT8 chain on the
    512 workload: within the quantisation-noise criterion of the oracle run
    with the same range finder."""
    c = workloads.CONFIGS["lramm_512"]
    A, B = workloads.operands("lramm_512")
    A32, B32 = A.astype(np.float32), B.astype(np.float32)
    m, k = A.shape
    n = B.shape[1]
    plan = L.Plan(m, n, k, c["r"], c["p"], c["q"], seed=workloads.SEED_SKETCH, prec=(1, 1, 1),
                  sketch=L.SKETCH_E4M3)
    ws = plan.workspace()
    D = np_(L.matmul(plan, dev(A32), dev(B32), ws=ws)).astype(np.float64)
    assert L.status_read(ws) == 0
    rf8 = oracle.sketch8.range_finder_e4m3
    ref_q = oracle.lramm.lramm(A32, B32, c["r"], c["p"], c["q"], workloads.SEED_SKETCH, (1, 1, 1), rf=rf8)
    ref_f = oracle.lramm.lramm(A32, B32, c["r"], c["p"], c["q"], workloads.SEED_SKETCH, (0, 0, 0), rf=rf8)
    exact = oracle.lramm.exact_product(A32, B32)
    noise = oracle.lramm.rel_fro(ref_q, ref_f)
    assert oracle.lramm.rel_fro(D, ref_q) <= 1.5 * noise
    err_gpu, err_orc = oracle.lramm.rel_fro(D, exact), oracle.lramm.rel_fro(ref_q, exact)
    assert abs(err_gpu - err_orc) <= 0.10 * err_orc


def test_e4m3_sketch_refused_where_not_offered(L):
    with pytest.raises(L.LrammError) as e:
        L.Plan(256, 256, 256, 16, 4, 1, sketch=L.SKETCH_E4M3, a_type=L.BF16)
    assert e.value.code == 2
    plan = L.Plan(256, 256, 256, 16, 4, 1, sketch=L.SKETCH_E4M3)
    X = torch.randn(256, 256, device="cuda")
    with pytest.raises(L.LrammError) as e:
        L.rf_forward(plan, X, X)
    assert e.value.code == 2


def test_lramm_4096_e4m3_sketch_full_size(L):
    """The 4096 workload (INT8 chain): the e4m3 range finder's error against
    the FP64 product within 5% of the TF32 range finder's (the INT8 chain's
    quantisation noise dominates both errors; two runs whose factors differ
    by rounding are two draws of it, a few percent apart)."""
    c = workloads.CONFIGS["lramm_4096"]
    A, B = workloads.device_operands("lramm_4096", "cuda")
    m, k = A.shape
    n = B.shape[1]
    exact = A.double() @ B.double()
    nrm = exact.norm()
    errs = {}
    for name, sk in (("tf32", L.SKETCH_TF32), ("e4m3", L.SKETCH_E4M3)):
        plan = L.Plan(m, n, k, c["r"], c["p"], c["q"], seed=workloads.SEED_SKETCH, prec=(1, 1, 1), sketch=sk)
        ws = plan.workspace()
        D = L.matmul(plan, A, B, ws=ws)
        assert L.status_read(ws) == 0
        errs[name] = ((D.double() - exact).norm() / nrm).item()
    assert errs["e4m3"] <= 1.05 * errs["tf32"], errs
