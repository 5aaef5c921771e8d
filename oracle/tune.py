"""FP64 oracle of LRAMM's parameter tuning (Sec. 3.5): the probe estimate of
the relative Frobenius error of a candidate, and the selection rule.

TEST INFRASTRUCTURE: part of the CPU oracle.  Only tests/, __graft_entry__.smoke()
and bench.py's CPU-baseline leg may import it; the product path never does.

Readings (Sec. 3.5 relates the running time to r and the bit widths and
recommends r near a tenth of the dimension with d2 = 4, d1 = d3 = 8; it
gives no procedure; each reading is listed in the design notes):
  * A candidate is a rank r and a bit-width triple (d1, d2, d3); its cost is
    its measured time on the device (the paper's complexity model orders the
    candidates the same way but ignores the hardware), its error the
    relative Frobenius error against A B.
  * The error is estimated with s Gaussian probe columns G (n x s, N(0,1)
    entries): e = ||(A B - D) G||_F / ||A B G||_F; since E ||X G||_F^2 =
    s ||X||_F^2 for any X, numerator and denominator estimate the two
    Frobenius norms without forming A B.
  * Selection: the fastest candidate whose estimated error is at most the
    target; when none is, the most accurate one.
"""
import numpy as np

F64 = np.float64


def probe_error(A, B, D, G):
    """||(A B - D) G||_F / ||A B G||_F in FP64 (A B G as A (B G))."""
    A = np.asarray(A, F64)
    B = np.asarray(B, F64)
    G = np.asarray(G, F64)
    ABG = A @ (B @ G)
    DG = np.asarray(D, F64) @ G
    return float(np.linalg.norm(ABG - DG) / np.linalg.norm(ABG))


def select(candidates, target):
    """candidates: dicts with 'err' and 'ms'.  The fastest with err <= target
    (ties: the more accurate, then the first listed); else the most accurate."""
    ok = [c for c in candidates if c["err"] <= target]
    if ok:
        return min(ok, key=lambda c: (c["ms"], c["err"]))
    return min(candidates, key=lambda c: c["err"])
