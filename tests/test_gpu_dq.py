"""Direct quantised products (Algorithm 2 on the full operands: the paper's
DQ8 / DQ4 comparators) through the C ABI against the oracle's QM.

The quantisation decisions are FP32 on both sides (per-row a_max of A,
per-column a_max of B, lambda by IEEE division, one FP32 multiply, RNE), the
integer sums exact: INT8 and INT4 outputs are bit-identical to
oracle.quant.qm; E4M3 sums are FP32 (tensor cores) vs exact (oracle).
"""
import numpy as np
import pytest

import oracle
from tests import elementwise as EW

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_16917_gb300 as L
    L.load()
    return L


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _ops(m, k, n, seed):
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((m, k)) * np.exp(rng.uniform(-2, 2, (m, 1)))).astype(np.float32)
    B = (rng.standard_normal((k, n)) * np.exp(rng.uniform(-2, 2, (1, n)))).astype(np.float32)
    return A, B


SHAPES = [(150, 200, 90), (257, 1000, 129), (64, 4096, 96), (1, 33, 1), (512, 512, 512)]


@pytest.mark.parametrize("m,k,n", SHAPES)
@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("per_row", [True, False])
def test_dq_integer_bit_exact(L, m, k, n, prec, per_row):
    A, B = _ops(m, k, n, m + k + n + prec)
    D = L.dq_matmul(dev(A), dev(B), prec=prec, per_row=per_row).cpu().numpy()
    ref = oracle.quant.qm(A, B, prec, 0 if per_row else 1)
    assert np.array_equal(D, ref)


@pytest.mark.parametrize("m,k,n", [(150, 200, 90), (512, 512, 512)])
def test_dq_e4m3(L, m, k, n):
    A, B = _ops(m, k, n, 7 + m)
    D = L.dq_matmul(dev(A), dev(B), prec=3).cpu().numpy().astype(np.float64)
    # identical e4m3 codes and scales; the GPU sums the k code products in
    # FP32: element by element within k u sum |cA cB| sA sB (+ 2u)
    ref, mag = EW.qm_terms(A, B, 3)
    bound = EW.qm_bound(mag, ref, k)
    assert np.all(np.abs(D - ref) <= bound)


def test_dq_alpha_beta(L):
    m, k, n = 200, 300, 180
    A, B = _ops(m, k, n, 9)
    C = np.random.default_rng(10).standard_normal((m, n)).astype(np.float32)
    D = L.dq_matmul(dev(A), dev(B), prec=1, alpha=0.5, beta=-2.0, C=dev(C)).cpu().numpy().astype(np.float64)
    qm = oracle.quant.qm(A, B, 1)
    v = (np.float32(0.5) * qm).astype(np.float32).astype(np.float64)
    ref = v - 2.0 * C.astype(np.float64)                 # one FMA after the dequantisation
    assert np.all(np.abs(D - ref) <= 2.0 ** -24 * np.abs(ref) + 1e-30)


def test_dq_error_within_elementwise_bound(L):
    """DQ8 against the exact product: within the elementwise bound the
    oracle's pins check (|a| e_b + e_a |b| + k e_a e_b, e = s/2)."""
    m, k, n = 128, 1024, 96
    A, B = _ops(m, k, n, 11)
    D = L.dq_matmul(dev(A), dev(B), prec=1).cpu().numpy().astype(np.float64)
    exact = A.astype(np.float64) @ B.astype(np.float64)
    ea = np.abs(A).max(axis=1, keepdims=True) / 127.0 / 2.0
    eb = np.abs(B).max(axis=0, keepdims=True) / 127.0 / 2.0
    bound = (np.abs(A) @ np.ones((k, 1))) * eb + ea * (np.ones((1, k)) @ np.abs(B)) + k * ea * eb
    assert np.all(np.abs(D - exact) <= bound * (1 + 1e-4) + 1e-6 * np.abs(exact).max())
