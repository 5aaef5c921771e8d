"""Algorithmic work that bench.py divides by measured kernel times (CPU)."""
import bench


def test_jacobi_flops_per_pair():
    """18 l flops per column pair with V accumulated (three inner products,
    two columns of M and of V rotated), 12 l in the M-only form."""
    l, sweeps = 272, [6, 6]
    pairs = l * (l - 1) / 2
    assert bench.jacobi_work(l, sweeps) == 6 * pairs * 18 * l
    assert bench.jacobi_work(l, sweeps, with_v=False) == 6 * pairs * 12 * l
    assert bench.jacobi_work(l, [5, 7]) == bench.jacobi_work(l, [6, 6])   # mean over the two operands


def test_m_only_variants():
    """Quantised chains (and lead / tail chains) up to l = 544 take the M-only
    small SVD inside lramm_matmul; the FP32 chain keeps V_s."""
    assert bench.m_only_svd("int8", 272) and bench.m_only_svd("e4m3", 144)
    assert bench.m_only_svd("lead64_mxfp4", 544) and bench.m_only_svd("884", 272)
    assert not bench.m_only_svd("fp32", 272)
    assert not bench.m_only_svd("int8", 576)
