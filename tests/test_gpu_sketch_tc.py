"""Range-finder products on the tcgen05 tensor cores (TF32) through the C ABI.

The operand X and the l-column matrix B enter the MMA as TF32 (10 explicit
mantissa bits); each product term then carries a relative error of at most
about 2^-10 (both inputs rounded or truncated), so every entry obeys
|out - X B| <= 2^-9 (|X| |B|) entrywise, FP32 accumulation error included.
The FP32 path through the same entry point is checked to 1e-6.
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


SHAPES = [(4096, 4096, 272), (700, 520, 64), (130, 1000, 8), (1000, 132, 144), (513, 2052, 400), (256, 256, 256)]


@pytest.mark.parametrize("rows,cols,l", SHAPES)
@pytest.mark.parametrize("transpose", [0, 1])
def test_sketch_product_tf32(L, rows, cols, l, transpose):
    rng = np.random.default_rng(rows + 3 * cols + 7 * l + transpose)
    X = rng.standard_normal((rows, cols)).astype(np.float32)
    B = rng.standard_normal((rows if transpose else cols, l)).astype(np.float32)
    out = L.sketch_product(torch.from_numpy(X).cuda(), torch.from_numpy(B).cuda(), transpose=bool(transpose),
                           sketch=L.SKETCH_TF32).cpu().numpy().astype(np.float64)
    Xd = X.astype(np.float64).T if transpose else X.astype(np.float64)
    ref = Xd @ B.astype(np.float64)
    mag = np.abs(Xd) @ np.abs(B.astype(np.float64))
    assert np.all(np.abs(out - ref) <= 2.0 ** -9 * mag), np.max(np.abs(out - ref) / mag)
    assert oracle.lramm.rel_fro(out, ref) < 2e-3


@pytest.mark.parametrize("transpose", [0, 1])
def test_sketch_product_fp32(L, transpose):
    rng = np.random.default_rng(5 + transpose)
    X = rng.standard_normal((333, 517)).astype(np.float32)
    B = rng.standard_normal((333 if transpose else 517, 37)).astype(np.float32)
    out = L.sketch_product(torch.from_numpy(X).cuda(), torch.from_numpy(B).cuda(), transpose=bool(transpose),
                           sketch=L.SKETCH_F32).cpu().numpy().astype(np.float64)
    ref = (X.astype(np.float64).T if transpose else X.astype(np.float64)) @ B.astype(np.float64)
    assert oracle.lramm.rel_fro(out, ref) < 1e-6


def test_sketch_product_tf32_rejects_unaligned_width(L):
    X = torch.zeros((64, 64), device="cuda")
    B = torch.zeros((64, 74), device="cuda")
    with pytest.raises(L.LrammError) as e:
        L.sketch_product(X, B, sketch=L.SKETCH_TF32)
    assert e.value.code == 2


def test_rsvd_with_tf32_sketch(L):
    """The whole range finder on tensor-core products: the rank-r
    approximation stays within a few TF32 roundings of the FP64 oracle."""
    m, k, r, p, q = 900, 700, 60, 8, 1
    X = workloads.lowrank(m, k, workloads.spectrum("exp32", min(m, k)), 77).astype(np.float32)
    plan = L.Plan(m, m, k, r, p, q, seed=7, sketch=L.SKETCH_TF32)
    ws = plan.workspace()
    U, S, V = (t.cpu().numpy() for t in L.rsvd(plan, 0, torch.from_numpy(X).cuda(), ws=ws))
    assert L.status_read(ws) == 0
    Uo, so, Vo = oracle.lramm.rsvd(X, r, p, q, 7, 0)
    err = oracle.lramm.rel_fro((U * S) @ V.T, (Uo * so) @ Vo.T)
    assert err < 4 * 2.0 ** -10, err


BF_SHAPES = [(4096, 4096, 272), (700, 520, 64), (130, 1000, 8), (1000, 136, 144), (513, 2056, 400), (600, 1200, 544),
             (256, 256, 1100)]


@pytest.mark.parametrize("rows,cols,l", BF_SHAPES)
@pytest.mark.parametrize("transpose", [0, 1])
@pytest.mark.parametrize("sketch", ["tf32", "bf16"])
def test_sketch_product_bf16_operand(L, rows, cols, l, transpose, sketch):
    """BF16 X is exact on the tensor cores; B enters as B_hi + B_lo (TF32
    mode: |B - B_hi - B_lo| <= 2^-16 |B|) or as B_hi (BF16 mode: 2^-9 |B|).
    l = 544 and 1100 run in column blocks of at most 512."""
    rng = np.random.default_rng(rows + 5 * cols + 11 * l + transpose)
    Xb = torch.from_numpy(rng.standard_normal((rows, cols)).astype(np.float32)).to(torch.bfloat16)
    X = Xb.float().numpy().astype(np.float64)
    B = rng.standard_normal((rows if transpose else cols, l)).astype(np.float32)
    mode = L.SKETCH_TF32 if sketch == "tf32" else L.SKETCH_BF16
    out = L.sketch_product(Xb.cuda(), torch.from_numpy(B).cuda(), transpose=bool(transpose),
                           sketch=mode).cpu().numpy().astype(np.float64)
    Xd = X.T if transpose else X
    ref = Xd @ B.astype(np.float64)
    mag = np.abs(Xd) @ np.abs(B.astype(np.float64))
    K = Xd.shape[1]
    rel = 2.0 ** -15 if sketch == "tf32" else 2.0 ** -8
    assert np.all(np.abs(out - ref) <= (rel + K * 2.0 ** -23) * mag), np.max(np.abs(out - ref) / mag)


@pytest.mark.parametrize("m,k,r,p,q", [(16384, 600, 128, 16, 2), (20000, 500, 60, 4, 0), (16400, 700, 256, 16, 1),
                                       (4096, 1000, 128, 16, 2), (3000, 800, 272, 16, 1), (2100, 900, 20, 8, 2)])
def test_rsvd_tf32_split_gram(L, m, k, r, p, q):
    """TF32 mode runs the CholeskyQR Grams of tall sketches (>= 2048 rows) in
    split TF32 on the tensor cores (l = 144, 64, 272, 288, 28; ragged row
    counts; l > 256 takes two MMA column groups): orthogonality to working
    precision after the two final passes, and the rank-r product within a
    few TF32 roundings."""
    X = workloads.lowrank(m, k, workloads.spectrum("poly1", min(m, k)), 88 + m).astype(np.float32)
    plan = L.Plan(m, m, k, r, p, q, seed=7, sketch=L.SKETCH_TF32)
    ws = plan.workspace()
    U, S, V = (t.cpu().numpy() for t in L.rsvd(plan, 0, torch.from_numpy(X).cuda(), ws=ws))
    assert L.status_read(ws) == 0
    Uo, so, Vo = oracle.lramm.rsvd(X, r, p, q, 7, 0)
    assert oracle.lramm.rel_fro((U * S) @ V.T, (Uo * so) @ Vo.T) < 4 * 2.0 ** -10
    tol = 4.0 * np.sqrt(max(m, k) * (r + p)) * 2.0 ** -24
    assert np.abs(U.T @ U - np.eye(r)).max() < 4 * tol
