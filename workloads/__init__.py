"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module only draws inputs; it contains none of LRAMM's arithmetic.  The
paper evaluates on synthetic random matrices (uniform, exponential, normal,
binary-uniform entries; Sec. 4.2-4.3); the workloads below stand in for them
with matrices of controlled singular-value decay, A = U diag(sigma) V^T with
Haar-random U, V (the Q factor of a seeded Gaussian, columns sign-fixed so
that diag(R) > 0).

Workload table (sizes, spectra, rank parameters):
  lramm_512      m=n=k=512,   FP32, sigma_i = exp(-i/32), plus 1e-6 N(0,1)
                 entrywise noise; r=64, p=10, q=1
  lramm_4096     m=n=k=4096,  FP32, sigma_i = (1+i)^-1; r=256, p=16, q=2
  lramm_8192     m=n=k=8192,  BF16, sigma_i = (1+i/16)^-2; r=512, p=32, q=1
  rf_linear      X 16384x4096 BF16 iid N(0,1); W 4096x11008 FP32,
                 sigma_i = exp(-i/128) + 1e-3; r=384, p=16, q=1
  lramm_32768    m=32768, k=4096, n=32768, FP32, sigma_i = (1+i)^-1.5;
                 r=128, p=16, q=2
  qsvd_4096      Algorithm 4 on one 4096 x 4096 FP32 matrix (the A of
                 lramm_4096: sigma_i = (1+i)^-1); r=256, p=16, q=2
Entry-distribution matrices (`entry_matrix`): the paper's precision tests
draw i.i.d. U(0,1), Exp(1), N(0,1) and Bernoulli(1/2) entries.
Seeds: A 1001, B 1002, X 1003, sketch 7.
"""
import numpy as np

SEED_A, SEED_B, SEED_X, SEED_SKETCH = 1001, 1002, 1003, 7

CONFIGS = {
    "lramm_512": dict(m=512, n=512, k=512, dtype="f32", spectrum="exp32",
                      noise=1e-6, r=64, p=10, q=1),
    "lramm_4096": dict(m=4096, n=4096, k=4096, dtype="f32", spectrum="poly1",
                       noise=0.0, r=256, p=16, q=2),
    "lramm_8192": dict(m=8192, n=8192, k=8192, dtype="bf16", spectrum="poly2_16",
                       noise=0.0, r=512, p=32, q=1),
    "rf_linear": dict(m=16384, n=11008, k=4096, dtype="bf16", spectrum="exp128",
                      noise=0.0, r=384, p=16, q=1),
    "lramm_32768": dict(m=32768, n=32768, k=4096, dtype="f32", spectrum="poly1.5",
                        noise=0.0, r=128, p=16, q=2),
    "qsvd_4096": dict(m=4096, n=4096, k=4096, dtype="f32", spectrum="poly1",
                      noise=0.0, r=256, p=16, q=2),
}


def spectrum(name, count):
    """Singular values sigma_0 .. sigma_{count-1} (index from 0, sigma_0 = 1)."""
    i = np.arange(count, dtype=np.float64)
    if name == "exp32":
        return np.exp(-i / 32.0)
    if name == "poly1":
        return (1.0 + i) ** -1.0
    if name == "poly2_16":
        return (1.0 + i / 16.0) ** -2.0
    if name == "exp128":
        return np.exp(-i / 128.0) + 1e-3
    if name == "poly1.5":
        return (1.0 + i) ** -1.5
    raise ValueError("unknown spectrum %r" % name)


def haar(rows, cols, rng):
    """rows x cols matrix with orthonormal columns, Haar-distributed (rows >= cols)."""
    G = rng.standard_normal((rows, cols))
    Q, R = np.linalg.qr(G, mode="reduced")
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d[None, :]


def lowrank(rows, cols, sigma, seed, noise=0.0):
    """U diag(sigma) V^T (+ noise * N(0,1) entrywise) in FP64, U, V Haar."""
    rng = np.random.default_rng(seed)
    p = min(rows, cols, len(sigma))
    U = haar(rows, p, rng)
    V = haar(cols, p, rng)
    X = (U * np.asarray(sigma[:p])[None, :]) @ V.T
    if noise:
        X = X + noise * rng.standard_normal((rows, cols))
    return X


def exact_rank(rows, cols, rank, seed, decay=0.5):
    """Matrix of exact rank `rank` with sigma_i = decay^i (i < rank)."""
    sig = decay ** np.arange(rank, dtype=np.float64)
    return lowrank(rows, cols, sig, seed)


def gaussian(rows, cols, seed):
    """i.i.d. N(0,1) entries (FP64)."""
    return np.random.default_rng(seed).standard_normal((rows, cols))


ENTRY_DISTS = ("uniform", "exponential", "normal", "binary")


def entry_matrix(dist, rows, cols, seed):
    """i.i.d. entries of the paper's precision tests (Sec. 4.2-4.3, Fig. 3):
    U(0,1), Exp(1), N(0,1) or Bernoulli(1/2) on {0, 1} (FP64)."""
    rng = np.random.default_rng(seed)
    if dist == "uniform":
        return rng.uniform(0.0, 1.0, (rows, cols))
    if dist == "exponential":
        return rng.exponential(1.0, (rows, cols))
    if dist == "normal":
        return rng.standard_normal((rows, cols))
    if dist == "binary":
        return rng.integers(0, 2, (rows, cols)).astype(np.float64)
    raise ValueError("unknown entry distribution %r" % dist)


def operands(name, scale=None):
    """(A, B) of a workload as FP64 numpy arrays.

    scale=(m, n, k) overrides the sizes (same spectrum rule), for small
    stand-ins of the large workloads.
    """
    c = CONFIGS[name]
    m, n, k = scale if scale is not None else (c["m"], c["n"], c["k"])
    if name == "rf_linear":
        A = gaussian(m, k, SEED_X)
        B = lowrank(k, n, spectrum(c["spectrum"], min(k, n)), SEED_B)
        return A, B
    A = lowrank(m, k, spectrum(c["spectrum"], min(m, k)), SEED_A, c["noise"])
    B = lowrank(k, n, spectrum(c["spectrum"], min(k, n)), SEED_B, c["noise"])
    return A, B


def device_operands(name, device, dtype=None, sizes=None):
    """(A, B) of a full-size workload generated on a torch device (FP32 or BF16).

    Uses the same seeded Gaussian draws as `operands` (numpy, host side) but
    forms the Haar factors with torch.linalg.qr on the device, so large
    workloads are generated in seconds.  Rounding differs from `operands` in
    the last bits; every comparison feeds the same generated tensors to both
    sides.
    """
    import torch

    c = CONFIGS[name]
    m, n, k = sizes if sizes is not None else (c["m"], c["n"], c["k"])
    tdt = dtype or (torch.bfloat16 if c["dtype"] == "bf16" else torch.float32)

    def haar_dev(rows, cols, rng):
        G = torch.from_numpy(rng.standard_normal((rows, cols)).astype(np.float32)).to(device)
        Q, R = torch.linalg.qr(G, mode="reduced")
        d = torch.sign(torch.diagonal(R))
        d[d == 0] = 1.0
        return Q * d[None, :]

    def lowrank_dev(rows, cols, sigma, seed, noise):
        rng = np.random.default_rng(seed)
        p = min(rows, cols)
        U = haar_dev(rows, p, rng)
        V = haar_dev(cols, p, rng)
        s = torch.from_numpy(np.asarray(sigma[:p], dtype=np.float32)).to(device)
        X = (U * s[None, :]) @ V.T
        if noise:
            X = X + noise * torch.from_numpy(
                rng.standard_normal((rows, cols)).astype(np.float32)).to(device)
        return X

    if name == "rf_linear":
        A = torch.from_numpy(gaussian(m, k, SEED_X).astype(np.float32)).to(device)
        B = lowrank_dev(k, n, spectrum(c["spectrum"], min(k, n)), SEED_B, 0.0)
    else:
        A = lowrank_dev(m, k, spectrum(c["spectrum"], min(m, k)), SEED_A, c["noise"])
        B = lowrank_dev(k, n, spectrum(c["spectrum"], min(k, n)), SEED_B, c["noise"])
    return A.to(tdt).contiguous(), B.to(tdt).contiguous()
