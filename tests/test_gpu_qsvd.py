"""Algorithm 4 (quantised SVD of one matrix) through the C ABI against the oracle.

Bars: the codes and scales of U~_k' and V_k' are bit-exact against the
oracle's quantiser applied to the factors the CUDA path quantised (returned
through Uf / Vf); those factors match the oracle's RSVD to the FP32 tolerance
of the RSVD tests; the approximation deq(U~') deq(V')^T is bit-exact against
fp32(fp32(acc) * fp32(su * sv)) for integer codes (exact integer sums) and
within K u sum |cu cv| su sv of the exact sum when E4M3 codes take part
(FP32 accumulation); Theorem 4.4's bound holds for the result.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests import pins

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

I8, I4, E4 = 1, 2, 3
# D of Theorem 4.4's |r| <= a_max / D per entry (the paper's 1 / lambda): the
# integer formats' 2^(d-1) - 1; for e4m3 the top binade [256, 448] has spacing
# 32, so a code is off by at most 16 / lambda = a_max / 28.
D_OF = {I8: 127.0, I4: 7.0, E4: 28.0}


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_16917_gb300 as L
    L.load()
    return L


def np_(t):
    return t.detach().cpu().numpy()


def codes_np(c):
    return c.float().cpu().numpy().astype(np.float64)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _plan(L, which, rows, cols, r, p, q, **kw):
    # which = 0: X is A (m x k); which = 1: X is B (k x n)
    if which == 0:
        return L.Plan(rows, cols, cols, r, p, q, seed=7, **kw)
    return L.Plan(rows, cols, rows, r, p, q, seed=7, **kw)


def _expected_xr(cu, su, cv, sv, pu, pv, per_row):
    """The product's reference: exact FP64 code sums; for integer codes the
    kernel's FP32 dequantisation order reproduced exactly."""
    acc = cu @ cv.T
    su = np.asarray(su, np.float32)
    sv = np.asarray(sv, np.float32)
    s = (su[:, None] * sv[None, :]) if per_row else np.full((1, 1), su[0] * sv[0], np.float32)
    exact = acc.astype(np.float32) * s.astype(np.float32)
    bound = np.abs(cu) @ np.abs(cv).T * s.astype(np.float64)
    return exact, acc, s.astype(np.float64), bound


def _check(L, X, which, r, p, q, pu, pv, scale, A_sigma=None):
    rows, cols = X.shape
    plan = _plan(L, which, rows, cols, r, p, q, scale=scale)
    per_row = scale == 0
    out = L.qsvd(plan, which, dev(X), pu, pv, factors=True)
    torch.cuda.synchronize()
    Uf, Vf = np_(out["Uf"]), np_(out["Vf"])
    Xr = np_(out["Xr"])
    # factors: the oracle's RSVD of the same input
    Ut_o, V_o, so = oracle.qsvd.factors(X, r, p, q, 7, which)
    Ak_o = Ut_o.astype(np.float64) @ V_o.astype(np.float64).T
    assert oracle.lramm.rel_fro(Uf.astype(np.float64) @ Vf.T.astype(np.float64), Ak_o) < 1e-5
    assert np.allclose(np.linalg.norm(Uf.astype(np.float64), axis=0), so[:r], rtol=1e-5, atol=1e-6 * so[0])
    # codes and scales: bit-exact against the oracle's quantiser on the same factors
    cu, cv = codes_np(out["Uc"]), codes_np(out["Vc"])
    for f, c, s, prec in ((Uf, cu, np_(out["Us"]), pu), (Vf, cv, np_(out["Vs"]), pv)):
        (oc, os_), _ = oracle.qsvd.quantise(f, prec, scale)
        assert np.array_equal(c[:, :r], oc)
        assert np.all(c[:, r:] == 0)
        assert np.array_equal(s, os_)
    # the approximation
    exact, acc, sc, bound = _expected_xr(cu, np_(out["Us"]), cv, np_(out["Vs"]), pu, pv, per_row)
    if E4 not in (pu, pv):
        assert np.array_equal(Xr, exact)
    else:
        kq = cu.shape[1]
        tol = kq * 2.0 ** -24 * bound + 2.0 ** -23 * np.abs(acc * sc)
        assert np.all(np.abs(Xr - acc * sc) <= tol + 1e-30)
    # Theorem 4.4 (n the larger dimension, r read as k)
    sig = A_sigma if A_sigma is not None else np.linalg.svd(X.astype(np.float64), compute_uv=False)
    err2 = np.linalg.norm(Xr.astype(np.float64) - X) ** 2
    assert err2 <= pins._thm44_rhs(sig, rows, cols, r, D_OF[pu], D_OF[pv])
    return out


PAIRS = [(I8, I8), (I8, I4), (I4, I8), (I4, I4), (E4, E4), (I4, E4), (E4, I4)]


@pytest.mark.parametrize("pu,pv", PAIRS)
@pytest.mark.parametrize("which", [0, 1])
def test_qsvd_small(L, pu, pv, which):
    X = workloads.lowrank(300, 260, workloads.spectrum("exp32", 260), 700).astype(np.float32)
    _check(L, X, which, 24, 8, 1, pu, pv, 0)


@pytest.mark.parametrize("pu,pv", [(I8, I4), (E4, E4), (I4, I4)])
def test_qsvd_per_tensor(L, pu, pv):
    X = workloads.entry_matrix("uniform", 280, 330, 701).astype(np.float32)
    _check(L, X, 0, 20, 8, 2, pu, pv, 1)


@pytest.mark.parametrize("pu,pv", [(I8, I8), (I8, I4), (E4, I4)])
def test_qsvd_several_tiles_ragged(L, pu, pv):
    """1000 x 700 at r = 100: 8 row tiles of 128 (the last one ragged), three
    column tiles, K = 128 (r padded with zero codes)."""
    X = workloads.lowrank(1000, 700, workloads.spectrum("poly1", 700), 702).astype(np.float32)
    _check(L, X, 0, 100, 12, 2, pu, pv, 0)


def test_qsvd_bf16_operand(L):
    """B side stored in bfloat16: the factors follow the oracle run on the
    bfloat16 values."""
    X = workloads.lowrank(400, 520, workloads.spectrum("poly2_16", 400), 703).astype(np.float32)
    Xb = torch.from_numpy(X).to(torch.bfloat16)
    Xv = Xb.float().numpy()
    plan = L.Plan(400, 520, 400, 32, 8, 1, seed=7, b_type=L.BF16)
    out = L.qsvd(plan, 1, Xb.cuda(), I8, I4, factors=True)
    Uf, Vf = np_(out["Uf"]), np_(out["Vf"])
    Ut_o, V_o, _ = oracle.qsvd.factors(Xv, 32, 8, 1, 7, 1)
    assert oracle.lramm.rel_fro(Uf.astype(np.float64) @ Vf.T, Ut_o.astype(np.float64) @ V_o.T) < 1e-5
    (oc, os_), _ = oracle.qsvd.quantise(Uf, I8, 0)
    assert np.array_equal(codes_np(out["Uc"])[:, :32], oc)
    (oc, os_), _ = oracle.qsvd.quantise(Vf, I4, 0)
    assert np.array_equal(codes_np(out["Vc"])[:, :32], oc)


def test_qsvd_exact_rank(L):
    """An exactly rank-k matrix: the unquantised factors reproduce it and the
    approximation error is the quantisation error alone, below its Theorem
    4.2 triangle bound."""
    rows, cols, k = 256, 192, 8
    X = workloads.exact_rank(rows, cols, k, 704).astype(np.float32)
    out = _check(L, X, 0, k, 8, 1, I8, I4, 0)
    Uf, Vf = np_(out["Uf"]).astype(np.float64), np_(out["Vf"]).astype(np.float64)
    assert oracle.lramm.rel_fro(Uf @ Vf.T, X) < 1e-5
    sig = np.linalg.svd(X.astype(np.float64), compute_uv=False)
    _, du = oracle.qsvd.quantise(np_(out["Uf"]), I8, 0)
    _, dv = oracle.qsvd.quantise(np_(out["Vf"]), I4, 0)
    nu, nv = np.linalg.norm(du - Uf), np.linalg.norm(dv - Vf)
    err = np.linalg.norm(np_(out["Xr"]) - X)
    assert err <= (np.linalg.norm(Uf @ Vf.T - X) + nu + sig[0] * nv + nu * nv) * (1 + 1e-5) + 1e-6


def test_qsvd_zero_matrix(L):
    """Degenerate input: a zero matrix gives zero factors, zero codes and
    scales and a zero approximation (no NaN / Inf)."""
    X = np.zeros((200, 150), np.float32)
    plan = _plan(L, 0, 200, 150, 16, 4, 1)
    ws = torch.empty(L.load().lramm_qsvd_ws_bytes(plan.handle, 0, I8, I4), dtype=torch.uint8, device="cuda")
    out = L.qsvd(plan, 0, dev(X), I8, I4, factors=True, ws=ws)
    assert L.status_read(ws) in (0, 5)
    for key in ("Uc", "Vc", "Us", "Vs", "Xr"):
        v = out[key].float().cpu().numpy()
        assert np.all(v == 0), key


def test_qsvd_codes_only(L):
    """Without Xr and factor outputs (and the INT8 / E4M3 pair, which has no
    code product) the codes are still those of the factors."""
    X = workloads.lowrank(300, 260, workloads.spectrum("exp32", 260), 705).astype(np.float32)
    plan = _plan(L, 0, 300, 260, 24, 8, 1)
    a = L.qsvd(plan, 0, dev(X), I8, E4, factors=True, reconstruct=False)
    b = L.qsvd(plan, 0, dev(X), I8, E4, factors=False, reconstruct=False)
    for key in ("Uc", "Vc", "Us", "Vs"):
        assert torch.equal(a[key].float(), b[key].float()), key
    (oc, _), _ = oracle.qsvd.quantise(np_(a["Vf"]), E4, 0)
    assert np.array_equal(codes_np(a["Vc"])[:, :24], oc)


def test_qsvd_full_size_lramm_4096(L):
    """The 4096 x 4096 operand at r = 256, p = 16, q = 2 (sigma_i = 1/(1+i)),
    INT8 / INT4: codes bit-exact on the returned factors, sampled entries of
    the approximation bit-exact, factors against the exact spectrum, and
    Theorem 4.4 with the workload's known singular values."""
    c = workloads.CONFIGS["lramm_4096"]
    A, _ = workloads.device_operands("lramm_4096", "cuda")
    m, k = A.shape
    r = c["r"]
    plan = L.Plan(m, c["n"], k, r, c["p"], c["q"], seed=workloads.SEED_SKETCH)
    out = L.qsvd(plan, 0, A, I8, I4, factors=True)
    torch.cuda.synchronize()
    Uf, Vf = np_(out["Uf"]), np_(out["Vf"])
    sig = workloads.spectrum(c["spectrum"], min(m, k))
    # leading singular values (the sketch's gap is wide there); the trailing
    # ones sit at a small spectral gap (sigma_272 / sigma_256 = 0.94)
    assert np.allclose(np.linalg.norm(Uf[:, :64].astype(np.float64), axis=0), sig[:64], rtol=2e-3)
    assert np.abs(Vf.astype(np.float64).T @ Vf - np.eye(r)).max() < 1e-4
    cu, cv = codes_np(out["Uc"]), codes_np(out["Vc"])
    for f, cc, s, prec in ((Uf, cu, np_(out["Us"]), I8), (Vf, cv, np_(out["Vs"]), I4)):
        (oc, os_), _ = oracle.qsvd.quantise(f, prec, 0)
        assert np.array_equal(cc[:, :r], oc)
        assert np.array_equal(s, os_)
    Xr = out["Xr"]
    rng = np.random.default_rng(11)
    ii = rng.integers(0, m, 4000)
    jj = rng.integers(0, k, 4000)
    su, sv = np_(out["Us"]), np_(out["Vs"])
    acc = np.einsum("st,st->s", cu[ii], cv[jj])
    ref = acc.astype(np.float32) * (su[ii] * sv[jj]).astype(np.float32)
    got = np_(Xr[torch.from_numpy(ii).cuda(), torch.from_numpy(jj).cuda()])
    assert np.array_equal(got, ref)
    err2 = float(torch.linalg.norm(Xr.double() - A.double()) ** 2)
    assert err2 <= pins._thm44_rhs(sig, m, k, r, 127.0, 7.0)
    # the error is dominated by the truncation (sum of sigma_i^2, i >= r) and INT4 on V
    tail = float(np.sum(sig[r:] ** 2))
    assert err2 >= tail * (1 - 1e-3)
