"""The shifted CholeskyQR fallback on a sketch too ill-conditioned for the
plain 4u shift (Sec. 2.2 asks for a Q with orthonormal columns).

Spectrum sigma_i = exp(-i/32) with l = r + p = 400 sketch columns: sigma_l /
sigma_1 ~ 4e-6, so the Gram's smallest eigenvalues sit far below the FP32
rounding of an l x l Cholesky and a pivot comes out non-positive.  The
library then refactors that Gram with a larger shift and, for the final
two-pass orthonormalisations, adds a third pass (shifted CholeskyQR3).
A Gram-based orthonormalisation in FP32 resolves directions down to about
sqrt(u) sigma_1 (2.4e-4 sigma_1, i ~ 267 here), so the rank is r = 160
(sigma_r ~ 6.7e-3 sigma_1) with a large oversampling p = 240.
Bars: status 0, the library's count of factorisations that broke down at
least 1 (the fallback ran), U and V orthonormal to ~sqrt(rows l) u, and the
rank-r product within the TF32 bar (4 x 2^-10) of the oracle's FP64
Householder range finder, or with FP32 products within 5e-5: the shifted
pass leaves Q1 with a condition number near 1 / sqrt(shift) ~ 50, so FP32
rounding of that pass reaches the subspace amplified by up to kappa sqrt(l)
u ~ 6e-5 (the plain passes' 1e-5 bar assumes kappa ~ 1).
"""
import numpy as np
import pytest

import oracle
import workloads
from tests.test_gpu_parity import quantised_agreement

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BRK_COUNT_WORD = 20   # status word 20 + side: factorisations of the call that broke down


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_16917_gb300 as L
    L.load()
    return L


@pytest.mark.parametrize("sketch", ["f32", "tf32"])
@pytest.mark.parametrize("which", [0, 1])
def test_rank_deficient_sketch_takes_shifted_cqr3(L, sketch, which):
    m, k, r, p, q = 1300, 1100, 160, 240, 1
    X = workloads.lowrank(m, k, workloads.spectrum("exp32", min(m, k)), 501).astype(np.float32)
    mode = L.SKETCH_TF32 if sketch == "tf32" else L.SKETCH_F32
    plan = L.Plan(m, m, k, r, p, q, seed=7, sketch=mode) if which == 0 else L.Plan(k, k, m, r, p, q, seed=7,
                                                                                      sketch=mode)
    ws = plan.workspace()
    U, S, V = (t.cpu().numpy() for t in L.rsvd(plan, which, torch.from_numpy(X).cuda(), ws=ws))
    info = L.info_read(ws, 24)
    assert L.status_read(ws) == 0
    if sketch == "f32":
        # FP32 products keep the trailing directions down to ~u: the Gram
        # breaks down; TF32 products (2^-11) leave a noise floor above the
        # shift and the plain passes factor (either way the bars below hold)
        assert info[BRK_COUNT_WORD + which] >= 1
    tol = 4.0 * np.sqrt(max(m, k) * (r + p)) * 2.0 ** -24
    assert np.abs(U.T @ U - np.eye(r)).max() < tol
    assert np.abs(V.T @ V - np.eye(r)).max() < tol
    Uo, so, Vo = oracle.lramm.rsvd(X, r, p, q, 7, which)
    bar = 5e-5 if sketch == "f32" else 4 * 2.0 ** -10
    assert oracle.lramm.rel_fro((U * S) @ V.T, (Uo * so) @ Vo.T) < bar


def test_rank_deficient_matmul_int8(L):
    """The same regime through lramm_matmul (INT8 chain, M-only small SVD:
    the fallback's third pass also updates R = L3^T L2^T L1^T)."""
    m, n, k, r, p, q = 1200, 1000, 1100, 160, 240, 1
    A = workloads.lowrank(m, k, workloads.spectrum("exp32", min(m, k)), 502).astype(np.float32)
    B = workloads.lowrank(k, n, workloads.spectrum("exp32", min(k, n)), 503).astype(np.float32)
    plan = L.Plan(m, n, k, r, p, q, seed=7, prec=(1, 1, 1))
    ws = plan.workspace()
    D = L.matmul(plan, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), ws=ws).cpu().numpy()
    info = L.info_read(ws, 24)
    assert L.status_read(ws) == 0
    assert info[BRK_COUNT_WORD] + info[BRK_COUNT_WORD + 1] >= 1
    fac = oracle.lramm.factors(A, B, r, p, q, 7)
    quantised_agreement(D.astype(np.float64), oracle.lramm.chain(*fac, (1, 1, 1)), oracle.lramm.chain(*fac, (0, 0, 0)),
                        oracle.lramm.exact_product(A, B))
