"""Checks that pin the CPU oracle to facts outside itself.

Each pin_* function raises AssertionError when the oracle disagrees with what
the paper, a closed form, a textbook bound or an independent library fixes.
They are called by the oracle tests and, against deliberately broken copies
of the oracle, by the mutation tests (which expect them to fail).
"""
import ctypes
import ctypes.util
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


# --------------------------------------------------------------------------
# Philox and the Gaussian test matrix
# --------------------------------------------------------------------------
def _curand_lib():
    cands = ["/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")]
    for c in cands:
        if c and os.path.exists(c) or (c and not c.startswith("/")):
            try:
                return ctypes.CDLL(c)
            except OSError:
                continue
    return None


def curand_host_philox_words(seed, n_words):
    """Words from cuRAND's host-side Philox4x32-10 generator (an independent
    library implementation of the same published generator)."""
    lib = _curand_lib()
    if lib is None:
        return None
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        return None
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        buf = (ctypes.c_uint * n_words)()
        assert lib.curandGenerate(gen, buf, ctypes.c_size_t(n_words)) == 0
        return np.frombuffer(buf, dtype=np.uint32).copy()
    finally:
        lib.curandDestroyGenerator(gen)


# cuRAND's host generator emits Philox block (counter n, subsequence s) at
# output position n * 65536 + s (ordering observed and fixed by this test).
CURAND_SUBSEQ_STRIDE = 65536


def pin_philox_curand(philox):
    """Oracle Philox words == cuRAND host Philox words for several counters,
    streams (subsequences) and 64-bit seeds."""
    checked = 0
    for seed in (0, 7, 0x123456789ABCDEF, 0xFFFFFFFF00000001):
        ref = curand_host_philox_words(seed, 4 * (3 * CURAND_SUBSEQ_STRIDE))
        if ref is None:
            raise RuntimeError("cuRAND host generator unavailable")
        ref = ref.reshape(-1, 4)
        for stream in (0, 1, 2, 5, 300, 65535):
            mine = philox.philox_words(seed, stream, 3)
            for n in range(3):
                got = ref[n * CURAND_SUBSEQ_STRIDE + stream]
                assert np.array_equal(mine[n], got), (seed, stream, n, mine[n], got)
                checked += 1
    return checked


def pin_gaussian_stats(philox, n=400_000):
    """Omega entries are N(0,1): KS test, moments, and the Box-Muller radius
    z0^2 + z1^2 ~ chi^2(2) (mean 2); pairs uncorrelated; streams independent."""
    from scipy import stats

    Om = philox.gaussian_matrix(12345, 0, n // 400, 400).astype(np.float64).ravel()
    assert abs(Om.mean()) < 5.0 / np.sqrt(Om.size), Om.mean()
    assert abs(Om.var() - 1.0) < 0.01, Om.var()
    assert stats.kstest(Om, "norm").pvalue > 1e-4
    z = Om.reshape(-1, 2)
    assert abs((z ** 2).sum(1).mean() - 2.0) < 0.03
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 0.01
    Om2 = philox.gaussian_matrix(12345, 1, n // 400, 400).astype(np.float64).ravel()
    assert abs(np.corrcoef(Om, Om2)[0, 1]) < 0.01
    # the fourth moment of N(0,1) is 3
    assert abs((Om ** 4).mean() - 3.0) < 0.08


def pin_box_muller_special(philox):
    """Closed forms of the transform: u1 = 1 gives z = 0; u2 near 1/4 puts the
    whole radius into z1; u2 near 1/2 gives z0 = -radius."""
    x = np.array([0xFFFFFFFF], dtype=np.uint32)          # u1 = 2^24 * 2^-24 = 1
    z0, z1 = philox.box_muller(x, np.array([12345], dtype=np.uint32))
    assert z0[0] == 0.0 and z1[0] == 0.0
    # x = 0 -> u1 = 2^-24 -> radius sqrt(48 ln 2)
    rad = np.sqrt(48.0 * np.log(2.0))
    y_quarter = np.array([((1 << 21) << 9)], dtype=np.uint32)          # y>>9 = 2^21 -> u2 = (2^22+1)/2^24
    z0, z1 = philox.box_muller(np.array([0], dtype=np.uint32), y_quarter)
    assert abs(z1[0] - rad) < 1e-5 and abs(z0[0]) < 1e-5
    y_half = np.array([((1 << 22) << 9)], dtype=np.uint32)             # u2 = (2^23+1)/2^24
    z0, z1 = philox.box_muller(np.array([0], dtype=np.uint32), y_half)
    assert abs(z0[0] + rad) < 1e-5 and abs(z1[0]) < 1e-5


# --------------------------------------------------------------------------
# Quantiser, e4m3 and QM
# --------------------------------------------------------------------------
def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([p.strip() for p in line.split("|")])
    return rows


def pin_quant_golden(quant):
    """Hand-worked examples of Eqs. (get_lambda) and (Quantization)."""
    for bits, xs, codes in _read_golden("quant_worked_example.txt"):
        prec = quant.PREC_INT8 if int(bits) == 8 else quant.PREC_INT4
        x = np.array([[float(v) for v in xs.split()]], dtype=np.float32)
        want = np.array([[float(v) for v in codes.split()]])
        got, lam, s = quant.quantize(x, prec, 1)
        assert np.array_equal(got, want), (bits, xs, got, want)


def e4m3_decode_all():
    """All finite e4m3 values from the bit-field definition (OCP OFP8)."""
    vals = []
    for code in range(256):
        sgn = -1.0 if code & 0x80 else 1.0
        e = (code >> 3) & 0xF
        m = code & 0x7
        if e == 15 and m == 7:
            continue                                    # NaN
        v = (m / 8.0) * 2.0 ** -6 if e == 0 else (1.0 + m / 8.0) * 2.0 ** (e - 7)
        vals.append(sgn * v)
    return np.array(sorted(set(vals)))


def pin_e4m3(quant):
    """Golden roundings, every representable value maps to itself, every
    midpoint of two neighbours goes to the one with even mantissa."""
    for x, want in _read_golden("e4m3_rounding.txt"):
        got = quant.round_e4m3(np.float32(float(x)))
        assert float(got) == float(want), (x, got, want)
    grid = e4m3_decode_all()
    assert grid.max() == 448.0 and np.min(grid[grid > 0]) == 2.0 ** -9
    assert np.array_equal(quant.round_e4m3(grid.astype(np.float32)), grid)
    pos = grid[grid >= 0]
    mids = (pos[:-1] + pos[1:]) / 2.0
    got = quant.round_e4m3(mids.astype(np.float32))
    for lo, hi, g in zip(pos[:-1], pos[1:], got):
        # even neighbour: its mantissa field (value / grid step) is even
        step = hi - lo
        lo_even = int(round(lo / step)) % 2 == 0
        assert g == (lo if lo_even else hi), (lo, hi, g)
    # nudged just off the midpoint, rounding goes to the nearer neighbour
    up = quant.round_e4m3((mids * (1 + 1e-6)).astype(np.float32))
    assert np.array_equal(up, pos[1:])


def pin_quant_bounds(quant, seed=5):
    """Thm 4.2, elementwise: |x - deq(q(x))| <= lambda^-1, here <= (1/2 + eps) s
    under round-to-nearest; codes symmetric (q(-x) = -q(x)); the group's
    largest magnitude maps to +-D; codes within +-D."""
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((37, 53)) * np.exp(rng.uniform(-4, 4, (37, 1)))).astype(np.float32)
    for prec, D in ((quant.PREC_INT8, 127), (quant.PREC_INT4, 7)):
        for axis in (1, 0, None):
            c, lam, s = quant.quantize(X, prec, axis)
            deq = quant.dequantize(c, s, axis)
            sb = s[:, None] if axis == 1 else (s[None, :] if axis == 0 else s[0])
            assert np.all(np.abs(X - deq) <= (0.5 + 1e-5) * sb + 1e-30)
            cn, _, _ = quant.quantize(-X, prec, axis)
            assert np.array_equal(cn, -c)
            assert np.abs(c).max() == D
            if axis == 1:
                idx = np.argmax(np.abs(X), axis=1)
                assert np.all(np.abs(c[np.arange(X.shape[0]), idx]) == D)
    # e4m3: relative error at most 2^-4 (3 mantissa bits) for normal values
    c, lam, s = quant.quantize(X, quant.PREC_E4M3, 1)
    y = X * lam[:, None]
    normal = np.abs(y) >= 2.0 ** -6
    assert np.all(np.abs(c - y)[normal] <= 2.0 ** -4 * np.abs(y)[normal] + 1e-7)


def pin_qm_bruteforce(quant, seed=6):
    """The code product equals a brute-force loop in Python integers, including
    the all-extreme worst case; QM equals the dequantised operands' product."""
    rng = np.random.default_rng(seed)
    for (M, K, N) in ((3, 5, 4), (6, 17, 5)):
        a = rng.integers(-127, 128, (M, K))
        b = rng.integers(-127, 128, (K, N))
        want = [[sum(int(a[i, t]) * int(b[t, j]) for t in range(K)) for j in range(N)] for i in range(M)]
        got = quant.code_product(a, b)
        assert np.array_equal(got, np.array(want, dtype=np.float64))
    a = np.full((2, 1024), 127.0)
    b = np.full((1024, 2), -127.0)
    b[::2] = 127.0
    got = quant.code_product(a, b)
    assert np.array_equal(got, np.zeros((2, 2)))
    got = quant.code_product(a, np.full((1024, 1), -127.0))
    assert got[0, 0] == -127 * 127 * 1024
    # QM == deq(L) @ deq(R) (scales attached to the right indices)
    L = (rng.standard_normal((9, 31)) * np.exp(rng.uniform(-3, 3, (9, 1)))).astype(np.float32)
    R = (rng.standard_normal((31, 7)) * np.exp(rng.uniform(-3, 3, (1, 7)))).astype(np.float32)
    for prec in (quant.PREC_INT8, quant.PREC_INT4, quant.PREC_E4M3):
        for scale, (al, ar) in ((quant.SCALE_ROWCOL, (1, 0)), (quant.SCALE_TENSOR, (None, None))):
            cl, _, sl = quant.quantize(L, prec, al)
            cr, _, sr = quant.quantize(R, prec, ar)
            ref = quant.dequantize(cl, sl, al).astype(np.float64) @ quant.dequantize(cr, sr, ar).astype(np.float64)
            got = quant.qm(L, R, prec, scale).astype(np.float64)
            assert np.allclose(got, ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max()), (prec, scale)


def pin_qm_error_bound(quant, seed=7):
    """Eq. (er_quant) / Thm 4.3 for per-tensor scales, plus its elementwise
    form: |C - C~|_ij <= sum_t |a_it| e_b + e_a |b_tj| + e_a e_b with
    e = s/2 the largest rounding error of each operand."""
    rng = np.random.default_rng(seed)
    m, k, n = 40, 64, 30
    A = rng.uniform(-1, 1, (m, k)).astype(np.float32)
    Bm = rng.uniform(-1, 1, (k, n)).astype(np.float32)
    C = A.astype(np.float64) @ Bm.astype(np.float64)
    for prec in (quant.PREC_INT8, quant.PREC_INT4):
        Ct = quant.qm(A, Bm, prec, quant.SCALE_TENSOR).astype(np.float64)
        D = 127.0 if prec == quant.PREC_INT8 else 7.0
        lam1 = D / np.abs(A).max()
        lam2 = D / np.abs(Bm).max()
        sig1 = np.linalg.norm(A, 2)
        gam1 = np.linalg.norm(Bm, 2)
        bound = k * (sig1 / lam2 * np.sqrt(n) + gam1 / lam1 * np.sqrt(m) + np.sqrt(m * n) / (lam1 * lam2))
        assert np.linalg.norm(C - Ct) <= bound
        ea, eb = 0.5 / lam1, 0.5 / lam2
        elem = np.abs(A).astype(np.float64) @ np.full((k, n), eb) + np.full((m, k), ea) @ np.abs(Bm) + k * ea * eb
        assert np.all(np.abs(C - Ct) <= elem * (1 + 1e-5) + 1e-6)


# --------------------------------------------------------------------------
# Randomized SVD
# --------------------------------------------------------------------------
def pin_orth(lr, seed=8):
    """orth(Y) is the unique thin QR factor: Q^T Q = I, Q^T Y upper triangular
    with positive diagonal, Y = Q (Q^T Y)."""
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((70, 12)) @ np.diag(np.logspace(0, -6, 12))
    Q = lr.orth(Y)
    R = Q.T @ Y
    assert np.abs(Q.T @ Q - np.eye(12)).max() < 1e-13
    assert np.abs(np.tril(R, -1)).max() < 1e-12 * np.abs(R).max()
    assert np.all(np.diag(R) > 0)
    assert np.abs(Q @ R - Y).max() < 1e-13 * np.abs(Y).max()


def pin_rsvd_exact_rank(lr, wl, seed=9):
    """A matrix of rank <= r is reproduced to 1e-12 (the sketch captures its
    range with probability 1), for q = 0, 1, 2, and the factors are
    orthonormal with descending positive singular values."""
    for (m, k, rank, r, p) in ((60, 45, 6, 6, 4), (40, 70, 5, 8, 3), (33, 33, 10, 10, 2)):
        A = wl.exact_rank(m, k, rank, seed)
        for q in (0, 1, 2):
            U, s, V = lr.rsvd(A, r, p, q, 77, 0)
            assert U.shape == (m, r) and V.shape == (k, r) and s.shape == (r,)
            assert lr.rel_fro((U * s) @ V.T, A) < 1e-12
            assert np.abs(U.T @ U - np.eye(r)).max() < 1e-12
            assert np.abs(V.T @ V - np.eye(r)).max() < 1e-12
            assert np.all(np.diff(s) <= 0) and s[-1] >= 0
            sv = np.linalg.svd(A, compute_uv=False)
            assert np.allclose(s[:rank], sv[:rank], rtol=1e-12, atol=0)


def pin_rsvd_full_sketch(lr, seed=10):
    """With l = min(m, k) the range is captured exactly and RSVD reduces to the
    exact truncated SVD (numpy's LAPACK SVD): singular values and the rank-r
    product agree to 1e-12 (Thm 3.1: error = sqrt(sum_{j>r} sigma_j^2))."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((50, 30)) @ np.diag(0.8 ** np.arange(30)) @ rng.standard_normal((30, 30))
    r = 7
    U, s, V = lr.rsvd(A, r, 30 - r, 0, 3, 0)
    Uf, sf, Vft = np.linalg.svd(A, full_matrices=False)
    assert np.allclose(s, sf[:r], rtol=1e-12)
    Ar = (Uf[:, :r] * sf[:r]) @ Vft[:r]
    assert np.abs((U * s) @ V.T - Ar).max() < 1e-12 * np.abs(A).max()
    err = np.linalg.norm(A - Ar)
    assert abs(err - np.sqrt(np.sum(sf[r:] ** 2))) < 1e-12 * np.linalg.norm(A)
    assert err <= sf[r] * np.sqrt(30 - r) + 1e-12          # Thm 3.1 bound


def pin_rsvd_bounds(lr, wl, trials=120):
    """Eckart-Young lower bound holds for every draw; the mean range error
    obeys Halko-Martinsson-Tropp Thm 10.5 (Frobenius, q = 0) and the paper's
    Eq. (rsvderror_z) (spectral, l = 2r, q = 0, 1); power iterations drive the
    error to the optimum."""
    m, k, r, p = 64, 48, 6, 6
    sig = (1.0 + np.arange(min(m, k))) ** -1.0
    A = wl.lowrank(m, k, sig, 2024)
    tail_f = np.sqrt(np.sum(sig[r:] ** 2))
    errs_f, errs_2 = {0: [], 1: []}, {0: [], 1: []}
    for q in (0, 1):
        for t in range(trials):
            Q = lr.range_finder(A, r + p, q, 1000 + t, 0)
            Res = A - Q @ (Q.T @ A)
            errs_f[q].append(np.linalg.norm(Res))
            errs_2[q].append(np.linalg.norm(Res, 2))
            U, s, V = lr.rsvd(A, r, p, q, 1000 + t, 0)
            assert np.linalg.norm(A - (U * s) @ V.T) >= tail_f * (1 - 1e-12)
    hmt_f = np.sqrt(1.0 + r / (p - 1.0)) * tail_f
    assert np.mean(errs_f[0]) <= hmt_f, (np.mean(errs_f[0]), hmt_f)
    for q in (0, 1):
        paper = (1.0 + 4.0 * np.sqrt(2.0 * min(m, k) / (r - 1.0))) ** (1.0 / (2 * q + 1)) * sig[r]
        assert np.mean(errs_2[q]) <= paper, (q, np.mean(errs_2[q]), paper)
    assert np.mean(errs_f[1]) < np.mean(errs_f[0])
    U, s, V = lr.rsvd(A, r, p, 6, 5, 0)
    assert np.linalg.norm(A - (U * s) @ V.T) <= tail_f * (1 + 1e-6)


# --------------------------------------------------------------------------
# LRAMM (Algorithm 3)
# --------------------------------------------------------------------------
def pin_lramm_exact(lr, wl, quant):
    """Exact rank-r operands and unquantised factors: D = A B to 1e-12; the
    alpha/beta form D = alpha A B + beta C."""
    m, k, n, r = 48, 40, 36, 6
    A = wl.exact_rank(m, k, r, 31)
    B = wl.exact_rank(k, n, r, 32)
    Cx = A @ B
    F = (quant.PREC_F32,) * 3
    # factors are stored in FP32, so compare the FP64 chain of the FP64 factors
    U, s, V = lr.rsvd(A, r, 3, 1, 7, 0)
    W, g, Z = lr.rsvd(B, r, 3, 1, 7, 1)
    D = (U * s) @ (V.T @ W) @ (g[:, None] * Z.T)
    assert lr.rel_fro(D, Cx) < 1e-12
    Dq = lr.lramm(A, B, r, 3, 1, 7, F)
    assert lr.rel_fro(Dq, Cx) < 1e-6
    C0 = np.random.default_rng(3).standard_normal((m, n))
    D2 = lr.lramm(A, B, r, 3, 1, 7, F, alpha=2.0, beta=-0.5, C=C0)
    assert np.allclose(D2, 2.0 * Dq - 0.5 * C0, rtol=1e-12, atol=1e-12)


def pin_lramm_factor_identity(lr, wl, quant):
    """Algorithm 3's factors satisfy U~ V^T = A_r and W Z~ = B_r, so the
    unquantised chain equals A_r B_r (FP32 storage of the factors only)."""
    m, k, n, r, p = 50, 44, 38, 7, 4
    A = wl.lowrank(m, k, 0.7 ** np.arange(min(m, k)), 41)
    B = wl.lowrank(k, n, 0.6 ** np.arange(min(k, n)), 42)
    U, s, V = lr.rsvd(A, r, p, 1, 9, 0)
    W, g, Z = lr.rsvd(B, r, p, 1, 9, 1)
    Ut, Vf, Wf, Zt = lr.factors(A, B, r, p, 1, 9)
    assert np.allclose(Ut.astype(np.float64) @ Vf.T, (U * s) @ V.T, atol=1e-6)
    assert np.allclose(Wf.astype(np.float64) @ Zt, (W * g) @ Z.T, atol=1e-6)
    D = lr.chain(Ut, Vf, Wf, Zt, (quant.PREC_F32,) * 3)
    ref = ((U * s) @ V.T) @ ((W * g) @ Z.T)
    assert lr.rel_fro(D, ref) < 2e-6


def pin_lramm_bit_ordering(lr, wl, quant):
    """Sec. 4.2: with about a tenth of the dimension as rank, 884 and 844 are
    more accurate than 444 on uniformly distributed matrices, and 888 is the
    most accurate of the quantised triples."""
    rng = np.random.default_rng(11)
    m = 160
    A = rng.uniform(0, 1, (m, m))
    B = rng.uniform(0, 1, (m, m))
    Cx = A @ B
    r = m // 10
    I8, I4 = quant.PREC_INT8, quant.PREC_INT4
    Ut, V, W, Zt = lr.factors(A, B, r, 8, 1, 13)
    err = {}
    for name, pr in (("888", (I8, I8, I8)), ("884", (I8, I8, I4)), ("844", (I8, I4, I4)), ("444", (I4, I4, I4))):
        err[name] = lr.rel_fro(lr.chain(Ut, V, W, Zt, pr), Cx)
    assert err["884"] < err["444"] and err["844"] < err["444"], err
    assert err["888"] <= min(err.values()) + 1e-12, err


# ---------------------------------------------------------------- range-finder form (oracle/rf.py)
def _rf_case(seed, m=7, k=10, n=9):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((m, k))
    W = rng.standard_normal((k, n))
    G = rng.standard_normal((m, n))
    return X, W, G


def pin_qr_adjoint_fd(rf, seed=31, h=1e-6):
    """d/dY <dQ, Q(Y)> by central differences against qr_adjoint."""
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((11, 4))
    dQ = rng.standard_normal((11, 4))
    Q, R = rf.qr_pos(Y)
    g = rf.qr_adjoint(Q, R, dQ)
    for _ in range(4):
        E = rng.standard_normal(Y.shape)
        fd = (np.sum(dQ * rf.qr_pos(Y + h * E)[0]) - np.sum(dQ * rf.qr_pos(Y - h * E)[0])) / (2 * h)
        assert abs(fd - np.sum(g * E)) <= 1e-7 * (1.0 + abs(fd)), (fd, np.sum(g * E))


def pin_rf_gradients_fd(rf, seed=32, h=1e-6):
    """Directional derivatives of L(X, W) = <G, X Q(W) Q(W)^T W> by central
    differences (Omega fixed) against rf_backward, q = 0, 1, 2."""
    X, W, G = _rf_case(seed)
    rng = np.random.default_rng(seed + 1)
    for q in (0, 1, 2):
        dX, dW = rf.rf_backward(X, W, G, 3, 2, q, 7)

        def L(Xv, Wv):
            return np.sum(G * rf.rf_forward(Xv, Wv, 3, 2, q, 7))
        for _ in range(3):
            EX = rng.standard_normal(X.shape)
            EW = rng.standard_normal(W.shape)
            fdx = (L(X + h * EX, W) - L(X - h * EX, W)) / (2 * h)
            fdw = (L(X, W + h * EW) - L(X, W - h * EW)) / (2 * h)
            assert abs(fdx - np.sum(dX * EX)) <= 1e-6 * (1.0 + abs(fdx)), (q, fdx, np.sum(dX * EX))
            assert abs(fdw - np.sum(dW * EW)) <= 1e-6 * (1.0 + abs(fdw)), (q, fdw, np.sum(dW * EW))


def pin_rf_exact_rank(rf, seed=33):
    """W of rank <= l: Q Q^T W = W, so the range-finder product is X W exactly."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((20, 30))
    W = rng.standard_normal((30, 4)) @ rng.standard_normal((4, 25))
    for q in (0, 1):
        C = rf.rf_forward(X, W, 4, 2, q, 7)
        assert np.linalg.norm(C - X @ W) <= 1e-12 * np.linalg.norm(X @ W)
    T, P, Q = rf.rf_factors(X, W, 4, 2, 1, 7)
    assert np.abs(Q.T @ Q - np.eye(6)).max() <= 1e-13


def pin_copyltu(rf, seed=34):
    M = np.random.default_rng(seed).standard_normal((5, 5))
    S = rf.copyltu(M)
    assert np.array_equal(S, S.T)
    assert np.array_equal(np.tril(S), np.tril(M))


# --------------------------------------------------------------------------
# MXFP4, split-precision residuals, lead / tail E3
# --------------------------------------------------------------------------
def e2m1_decode_all():
    """All 16 e2m1 codes from the bit fields (1 sign, 2 exponent bits with
    bias 1, 1 mantissa bit): (value, mantissa bit)."""
    out = []
    for code in range(16):
        sgn = -1.0 if code & 8 else 1.0
        e = (code >> 1) & 3
        m = code & 1
        v = (m / 2.0) if e == 0 else (1.0 + m / 2.0) * 2.0 ** (e - 1)
        out.append((sgn * v, m))
    return out


def pin_e2m1(mixed):
    """Every representable value maps to itself; every midpoint of two
    neighbours goes to the one whose mantissa bit is 0; nudged midpoints go
    to the nearer one; magnitudes above 6 saturate; brute-force nearest-even
    on random values."""
    grid = sorted({v for v, _ in e2m1_decode_all() if v >= 0})
    assert grid == [0.0, 0.5, 1.0, 1.5, 2.0, 3.0, 4.0, 6.0]
    mant = {abs(v): m for v, m in e2m1_decode_all()}
    g = np.array(grid)
    assert np.array_equal(mixed.round_e2m1(g), g) and np.array_equal(mixed.round_e2m1(-g), -g)
    for lo, hi in zip(grid[:-1], grid[1:]):
        mid = (lo + hi) / 2.0
        want = lo if mant[lo] == 0 else hi
        assert mixed.round_e2m1(np.array([mid]))[0] == want, (lo, hi)
        assert mixed.round_e2m1(np.array([mid * (1 + 1e-9)]))[0] == hi
        assert mixed.round_e2m1(np.array([mid * (1 - 1e-9)]))[0] == lo
    assert mixed.round_e2m1(np.array([7.9, 100.0, -6.5]))[0] == 6.0
    rng = np.random.default_rng(41)
    v = rng.uniform(-6, 6, 5000)
    got = mixed.round_e2m1(v)
    d = np.abs(np.abs(v)[:, None] - g[None, :])
    best = g[np.argmin(d, axis=1)]
    assert np.array_equal(np.abs(got), best) and np.all(np.sign(got[got != 0]) == np.sign(v[got != 0]))


def pin_mx_scale_rule(mixed):
    """e = ceil(log2(amax / 6)): amax / 2^e lies in (3, 6] (no element
    saturates, the block's largest element uses the top binade), checked on
    random magnitudes and the power-of-two edges; a zero block gets -127."""
    rng = np.random.default_rng(42)
    amax = np.exp(rng.uniform(-30, 30, 20000)).astype(np.float32)
    edges = np.array([6.0, 3.0, 12.0, 1.5, 6.0 * 2.0 ** -20, 3.0 * 2.0 ** 10, 6.0000005, 2.9999998],
                     dtype=np.float32)
    amax = np.concatenate([amax, edges])
    e = mixed.mx_exponent(amax)
    ratio = amax.astype(np.float64) / np.exp2(e.astype(np.float64))
    assert np.all(ratio > 3.0) and np.all(ratio <= 6.0 * (1 + 2.0 ** -23))
    assert np.array_equal(mixed.mx_exponent(np.array([6.0, 3.0, 12.0], np.float32)), [0, -1, 1])
    assert mixed.mx_exponent(np.array([0.0], np.float32))[0] == -127


def pin_mxfp4_quantise(mixed, seed=43):
    """Block quantisation: |x - deq| <= half the grid step at |x| / 2^e
    times 2^e (<= 2^e overall), codes on the grid, block scales from each
    block's own amax (a large value in one block does not coarsen its
    neighbours), K tails shorter than a block."""
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((9, 77)) * np.exp(rng.uniform(-5, 5, (9, 77)))).astype(np.float32)
    X[2, 40] = 1e6
    c, e = mixed.quantize_mxfp4(X)
    assert c.shape == X.shape and e.shape == (9, 3)
    grid = np.array([0.0, 0.5, 1.0, 1.5, 2.0, 3.0, 4.0, 6.0])
    assert np.all(np.isin(np.abs(c), grid))
    deq = mixed.dequantize_mxfp4(c, e)
    scale = np.repeat(np.exp2(e.astype(np.float64)), 32, axis=1)[:, :77]
    y = np.abs(X) / scale
    half_step = np.where(y < 2, 0.25, np.where(y < 4, 0.5, 1.0))
    assert np.all(np.abs(X - deq) <= half_step * scale * (1 + 1e-12))
    for b in range(3):
        blk = X[:, 32 * b:32 * (b + 1)]
        assert np.array_equal(e[:, b], mixed.mx_exponent(np.max(np.abs(blk), axis=1)))


def pin_mx_product_bruteforce(mixed, seed=44):
    """The block-scaled product equals a Python loop over K of the
    dequantised elements (exact dyadic arithmetic), K tail included."""
    rng = np.random.default_rng(seed)
    L = (rng.standard_normal((3, 70)) * np.exp(rng.uniform(-3, 3, (3, 70)))).astype(np.float32)
    R = (rng.standard_normal((70, 4)) * np.exp(rng.uniform(-3, 3, (70, 4)))).astype(np.float32)
    cl, el = mixed.quantize_mxfp4(L)
    cr, er = mixed.quantize_mxfp4(R.T)
    got = mixed.mx_product(cl, el, cr, er)
    for i in range(3):
        for j in range(4):
            want = 0.0
            for k in range(70):
                want += (cl[i, k] * 2.0 ** int(el[i, k // 32])) * (cr[j, k] * 2.0 ** int(er[j, k // 32]))
            assert got[i, j] == want, (i, j, got[i, j], want)
    assert np.array_equal(mixed.qm_mxfp4(L, R), got.astype(np.float32))


def pin_hilo_residual(mixed, quant, seed=45):
    """The split-precision pair reconstructs x to half a lo step: |x -
    deq(hi) - deq(lo)| <= (1/2 + eps) s_lo + FP32 rounding; the residual's
    scale is at most about s_hi / (2 D)."""
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((33, 64)) * np.exp(rng.uniform(-3, 3, (33, 1)))).astype(np.float32)
    for prec, D in ((quant.PREC_INT8, 127.0), (quant.PREC_INT4, 7.0)):
        for axis in (1, 0, None):
            (ch, sh), (cl, sl) = mixed.quantize_hilo(X, prec, axis)
            rec = quant.dequantize(ch, sh, axis).astype(np.float64) + quant.dequantize(cl, sl, axis)
            sb = sl[:, None] if axis == 1 else (sl[None, :] if axis == 0 else sl[0])
            xb = np.abs(X).max(axis=1, keepdims=True) if axis == 1 else (
                np.abs(X).max(axis=0, keepdims=True) if axis == 0 else np.abs(X).max())
            assert np.all(np.abs(X - rec) <= (0.5 + 1e-5) * sb + 2.0 ** -23 * xb)
            assert np.all(sl <= (0.5 + 1e-5) * sh / D + 2.0 ** -23 * np.asarray(sh) * D)


def pin_lead_tail(mixed, quant, seed=46):
    """Reductions and accuracy of the lead / tail E3:
    lead = 0 is the plain QM in the tail precision; lead = r without
    residual is the plain QM in the lead precision; each residual term
    shrinks the lead block's error against the FP64 product (the split
    error is a small fraction of the unsplit one)."""
    rng = np.random.default_rng(seed)
    m, r, n = 40, 24, 36
    Ut = (rng.standard_normal((m, r)) * np.exp(-np.arange(r) / 6.0)).astype(np.float32)
    E2 = rng.standard_normal((r, n)).astype(np.float32)
    for tail in (quant.PREC_INT4, mixed.PREC_MXFP4):
        got = mixed.e3_lead_tail(Ut, E2, tail, 0, quant.PREC_INT8, 2)
        assert np.array_equal(got, mixed.qm_any(Ut, E2, tail, quant.SCALE_ROWCOL).astype(np.float64))
    got = mixed.e3_lead_tail(Ut, E2, quant.PREC_INT4, r, quant.PREC_INT8, 0)
    assert np.array_equal(got, quant.qm(Ut, E2, quant.PREC_INT8).astype(np.float64))
    exact = Ut.astype(np.float64) @ E2.astype(np.float64)
    errs = [np.linalg.norm(mixed.e3_lead_tail(Ut, E2, quant.PREC_INT4, r, quant.PREC_INT8, s) - exact)
            for s in (0, 1, 2)]
    assert errs[1] < 0.6 * errs[0] and errs[2] < 0.05 * errs[0], errs
    # split = 2 leaves only the lo.lo term and the lo roundings: ~ (s_lo / 2)-sized errors
    (uh, suh), (ul, sul) = mixed.quantize_hilo(Ut, quant.PREC_INT8, 1)
    (eh, seh), (el, sel) = mixed.quantize_hilo(E2, quant.PREC_INT8, 0)
    du = Ut.astype(np.float64) - quant.dequantize(uh, suh, 1) - quant.dequantize(ul, sul, 1)
    de = E2.astype(np.float64) - quant.dequantize(eh, seh, 0) - quant.dequantize(el, sel, 0)
    lolo = quant.dequantize(ul, sul, 1).astype(np.float64) @ quant.dequantize(el, sel, 0)
    bound = (np.abs(du) @ np.abs(E2) + np.abs(Ut) @ np.abs(de) + np.abs(lolo) + np.abs(du) @ np.abs(de))
    full = mixed.e3_lead_tail(Ut, E2, quant.PREC_INT4, r, quant.PREC_INT8, 2)
    assert np.all(np.abs(full - exact) <= bound * (1 + 1e-4) + 1e-6 * np.abs(exact).max())


# --------------------------------------------------------------------------
# Algorithm 4: quantised SVD of one matrix, Theorem 4.4
# --------------------------------------------------------------------------
def pin_qsvd_unquantised(qs, lr, wl, quant):
    """Without quantisation Algorithm 4's approximation is U~_k V_k^T, the
    rank-k RSVD: a matrix of exact rank k is reproduced (to the FP32 storage
    of the factors), the columns of U~_k = U_k Sigma_k have norms sigma_i,
    V_k has orthonormal columns, and with a full sketch (l = min(m, n)) the
    approximation is the truncated SVD of Eckart-Young (numpy's LAPACK)."""
    F = quant.PREC_F32
    for (m, n, k, p) in ((60, 45, 6, 4), (40, 70, 5, 3)):
        A = wl.exact_rank(m, n, k, 91)
        sv = np.linalg.svd(A, compute_uv=False)
        for q in (0, 1):
            _, _, Ap, s = qs.qsvd(A, k, p, q, 5, 0, F, F)
            assert Ap.shape == A.shape
            assert lr.rel_fro(Ap, A) < 1e-6
            Ut, V, _ = qs.factors(A, k, p, q, 5, 0)
            assert np.allclose(np.linalg.norm(Ut.astype(np.float64), axis=0), sv[:k], rtol=1e-6)
            assert np.abs(V.astype(np.float64).T @ V - np.eye(k)).max() < 1e-6
    rng = np.random.default_rng(92)
    A = rng.standard_normal((36, 28))
    k = 9
    _, _, Ap, _ = qs.qsvd(A, k, 28 - k, 0, 3, 0, F, F)
    Uf, sf, Vft = np.linalg.svd(A, full_matrices=False)
    Ak = (Uf[:, :k] * sf[:k]) @ Vft[:k]
    assert np.abs(Ap - Ak).max() < 1e-5 * np.abs(A).max()


def _rne(y):
    """Round half to even on a Python float (Python's round is half-even)."""
    return float(round(y))


def pin_qsvd_codes_bruteforce(qs, quant, seed=93):
    """The quantised factors carry Eq. (Quantization) codes of the rows of
    U~_k and V_k (scalar loops: a_max per row or per factor, lambda =
    fp32(D / a_max), code = round-half-even(fp32(x lambda)) clamped to D,
    scale fp32(a_max / D)), a row's largest code is D, and A' is the plain
    product of the dequantised factors (Quant~(Quant(.), T_F) then U~' V'^T)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((23, 17)) * np.linspace(0.5, 3.0, 17)[None, :]
    I8, I4 = quant.PREC_INT8, quant.PREC_INT4
    k, p, q = 5, 3, 1
    Ut, V, _ = qs.factors(A, k, p, q, 4, 0)
    for scale in (quant.SCALE_ROWCOL, quant.SCALE_TENSOR):
        for d1, d2 in ((I8, I4), (I4, I8)):
            (cu, su), (cv, sv), Ap, _ = qs.qsvd(A, k, p, q, 4, 0, d1, d2, scale)
            deq = []
            for M, codes, scales, prec in ((Ut, cu, su, d1), (V, cv, sv, d2)):
                D = np.float32(127.0 if prec == I8 else 7.0)
                rows = M.shape[0]
                if scale == quant.SCALE_TENSOR:
                    amaxes = [max(abs(float(x)) for x in M.ravel())] * rows
                else:
                    amaxes = [max(abs(float(x)) for x in M[i]) for i in range(rows)]
                out = np.zeros(M.shape)
                for i in range(rows):
                    am = np.float32(amaxes[i])
                    lam = np.float32(D / am)
                    s_i = np.float32(am / D)
                    assert np.float32(scales[0 if scale == quant.SCALE_TENSOR else i]) == s_i
                    for t in range(k):
                        y = float(np.float32(np.float32(M[i, t]) * lam))
                        c = min(max(_rne(y), -float(D)), float(D))
                        assert codes[i, t] == c, (i, t, codes[i, t], c)
                        out[i, t] = float(np.float32(np.float32(c) * s_i))
                    if scale == quant.SCALE_ROWCOL:
                        assert max(abs(codes[i])) == float(D)
                if scale == quant.SCALE_TENSOR:
                    assert np.abs(codes).max() == float(D)
                deq.append(out)
            ref = np.array([[sum(deq[0][i, t] * deq[1][j, t] for t in range(k))
                             for j in range(V.shape[0])] for i in range(Ut.shape[0])])
            assert np.allclose(Ap, ref, rtol=1e-12, atol=1e-14)


def _thm44_rhs(sig, m, n, k, D1, D2):
    """Theorem 4.4's right-hand side, n the larger dimension, r read as k."""
    nn = max(m, n)
    s1 = sig[0] ** 2
    tail = sig[k] ** 2 * (nn - k) if k < len(sig) else 0.0
    return (tail + m * k * s1 / D1 ** 2 + n * k * s1 / D2 ** 2
            + m * n * k * s1 / (D1 ** 2 * D2 ** 2))


def pin_qsvd_error_bounds(qs, wl, quant):
    """Theorem 4.2 per factor and Theorem 4.4 for the approximation.

    |U~_k' - U~_k|_F <= sqrt(m k) / lambda_1 with lambda_1 >= D1 / sigma_1
    (entries of U~ are at most sigma_1), and half of it for round-to-nearest;
    |V_k' - V_k|_F <= sqrt(n k) / (2 D2) (entries of V at most 1); the
    approximation error obeys the triangle inequality over the three error
    terms of the proof and Theorem 4.4's bound.  An exactly rank-k matrix
    (sigma_{k+1} = 0) keeps only the quantisation terms and its error is not
    zero."""
    I8, I4 = quant.PREC_INT8, quant.PREC_INT4
    rng = np.random.default_rng(94)
    cases = [("normal", rng.standard_normal((72, 90)), 12),
             ("uniform", rng.uniform(0.0, 1.0, (90, 64)), 10),
             ("decay", wl.lowrank(80, 80, 0.85 ** np.arange(80), 95), 14),
             ("rank6", wl.exact_rank(64, 50, 6, 96), 6)]
    for name, A, k in cases:
        m, n = A.shape
        sig = np.linalg.svd(A, compute_uv=False)
        Ut, V, _ = qs.factors(A, k, 6, 2, 8, 0)
        Ak = Ut.astype(np.float64) @ V.astype(np.float64).T
        for d1, d2 in ((I8, I8), (I8, I4), (I4, I8), (I4, I4)):
            D1 = 127.0 if d1 == I8 else 7.0
            D2 = 127.0 if d2 == I8 else 7.0
            _, du = qs.quantise(Ut, d1, quant.SCALE_ROWCOL)
            _, dv = qs.quantise(V, d2, quant.SCALE_ROWCOL)
            _, _, Ap, _ = qs.qsvd(A, k, 6, 2, 8, 0, d1, d2)
            RU = du - Ut.astype(np.float64)
            RV = dv - V.astype(np.float64)
            nu, nv = np.linalg.norm(RU), np.linalg.norm(RV)
            assert nu <= np.sqrt(m * k) * sig[0] / D1 * (0.5 + 1e-6), (name, d1, nu)
            assert nv <= np.sqrt(n * k) / D2 * (0.5 + 1e-6), (name, d2, nv)
            err = np.linalg.norm(Ap - A)
            tri = (np.linalg.norm(A - Ak) + nu + np.linalg.norm(Ut.astype(np.float64), 2) * nv + nu * nv)
            assert err <= tri * (1 + 1e-9), (name, d1, d2, err, tri)
            assert err ** 2 <= _thm44_rhs(sig, m, n, k, D1, D2), (name, d1, d2, err ** 2)
            if name == "rank6":
                assert err > 1e-4 * np.linalg.norm(A)
                assert np.linalg.norm(A - Ak) < 1e-6 * np.linalg.norm(A)
            if name == "normal":
                # round-to-nearest leaves errors uniform on half a step:
                # E |r|^2 = step^2 / 12 per entry, step = a_max(row) / D
                for M, Dq, prec in ((Ut, D1, d1), (V, D2, d2)):
                    (c, s), dq = qs.quantise(M, prec, quant.SCALE_ROWCOL)
                    model = np.sum(np.asarray(s, np.float64) ** 2) * k / 12.0
                    ratio = np.sum((dq - M.astype(np.float64)) ** 2) / model
                    assert 0.7 < ratio < 1.3, (name, prec, ratio)


# --------------------------------------------------------------------------
# E4M3 range finder (products of the range finder on e4m3 codes)
# --------------------------------------------------------------------------
def pin_rf_e4m3_structure(s8, lr, wl):
    """With the exact product in place of the quantised one, the e4m3 range
    finder is the range finder of Sec. 2.2 (same steps in the same order):
    identical bases."""
    A = wl.lowrank(60, 45, 0.8 ** np.arange(45), 71)
    for q in (0, 1, 2):
        Q1 = s8.range_finder_e4m3(A, 12, q, 5, 0, product=np.matmul)
        Q2 = lr.range_finder(A, 12, q, 5, 0)
        assert np.array_equal(Q1, Q2)


def pin_rf_e4m3_product(s8, quant, seed=72):
    """One quantised product by scalar loops: e4m3 codes of the rows of L and
    the columns of R (lambda = fp32(448 / a_max), code = e4m3(fp32(x lambda))),
    the exact code sum, then fp32(fp32(acc) * fp32(sL * sR))."""
    rng = np.random.default_rng(seed)
    L = rng.standard_normal((5, 7)) * np.exp(rng.uniform(-3, 3, (5, 1)))
    R = rng.standard_normal((7, 4)) * np.exp(rng.uniform(-3, 3, (1, 4)))
    got = s8.qproduct_e4m3(L, R)
    D = np.float32(448.0)

    def codes(v):
        v = [np.float32(x) for x in v]
        am = np.float32(max(abs(x) for x in v))
        lam = np.float32(D / am)
        return [float(quant.round_e4m3(np.float32(x * lam))) for x in v], np.float32(am / D)
    for i in range(5):
        cl, sl = codes(L[i])
        for j in range(4):
            cr, sr = codes(R[:, j])
            acc = sum(a * b for a, b in zip(cl, cr))
            want = float(np.float32(np.float32(acc) * np.float32(sl * sr)))
            assert got[i, j] == want, (i, j, got[i, j], want)


def pin_rf_e4m3_accuracy(s8, lr, wl):
    """The e4m3 range finder keeps the randomized SVD close to the FP64 one:
    Q orthonormal, and the rank-r error between the Eckart-Young floor and
    1.01 times the FP64 range finder's (decaying spectra, q = 1, 2)."""
    for (m, n, spec, r, p) in ((400, 300, (1.0 + np.arange(300)) ** -1.0, 32, 8),
                               (300, 360, np.exp(-np.arange(300) / 24.0), 24, 8)):
        A = wl.lowrank(m, n, spec, 73)
        floor = np.sqrt(np.sum(spec[r:] ** 2))
        for q in (1, 2):
            Q = s8.range_finder_e4m3(A, r + p, q, 9, 0)
            assert np.abs(Q.T @ Q - np.eye(r + p)).max() < 1e-12
            U, s, V = s8.rsvd_e4m3(A, r, p, q, 9, 0)
            U0, s0, V0 = lr.rsvd(A, r, p, q, 9, 0)
            e8 = np.linalg.norm(A - (U * s) @ V.T)
            e0 = np.linalg.norm(A - (U0 * s0) @ V0.T)
            assert floor * (1 - 1e-9) <= e8 <= 1.01 * e0, (m, q, e8, e0, floor)


# --------------------------------------------------------------------------
# Parameter tuning (Sec. 3.5): probe error estimate and selection
# --------------------------------------------------------------------------
def pin_probe_error(tn, seed=81):
    """E ||X G||_F^2 = s ||X||_F^2: with many probe columns the estimate
    converges to the exact relative Frobenius error (within 3%), with one
    probe it is a single draw of it; D = A B gives 0 (to rounding)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((60, 40))
    B = rng.standard_normal((40, 50))
    D = A @ B + 0.05 * rng.standard_normal((60, 50)) * np.abs(A @ B).mean()
    exact = np.linalg.norm(A @ B - D) / np.linalg.norm(A @ B)
    G = rng.standard_normal((50, 4000))
    est = tn.probe_error(A, B, D, G)
    assert abs(est - exact) <= 0.03 * exact, (est, exact)
    assert tn.probe_error(A, B, A @ B, G[:, :8]) < 1e-14
    # the estimate is invariant to the scale of the probes
    assert np.isclose(tn.probe_error(A, B, D, 3.0 * G[:, :16]), tn.probe_error(A, B, D, G[:, :16]), rtol=1e-12)


def pin_select(tn):
    """The selection rule on hand-made tables."""
    c = [dict(name="a", err=0.05, ms=2.5), dict(name="b", err=0.02, ms=4.0), dict(name="c", err=0.2, ms=1.0),
         dict(name="d", err=0.02, ms=3.0)]
    assert tn.select(c, 0.1)["name"] == "a"          # fastest within the target
    assert tn.select(c, 0.03)["name"] == "d"         # b and d qualify: the faster
    assert tn.select(c, 0.5)["name"] == "c"
    assert tn.select(c, 0.001)["name"] == "b"        # none qualifies: the most accurate (first of the ties)
    c2 = [dict(name="x", err=0.01, ms=2.0), dict(name="y", err=0.005, ms=2.0)]
    assert tn.select(c2, 0.02)["name"] == "y"        # equal times: the more accurate
