"""The element-wise bound helpers (tests/elementwise.py) against brute force:
values moved by less than their boundary distance keep their code, the
chain helper reproduces the oracle's chain, and a planted wrong term in a
lead / tail E3 exceeds its bound (CPU only)."""
import numpy as np
import pytest

import oracle
from tests import elementwise as EW

Q = oracle.quant


@pytest.mark.parametrize("prec", [Q.PREC_INT8, Q.PREC_E4M3])
def test_boundary_distance_keeps_codes(prec):
    rng = np.random.default_rng(3 + prec)
    a = np.abs(rng.standard_normal(50000) * np.exp(rng.uniform(-10, 6, 50000)))
    a = np.concatenate([a, [0.0, 1.0, 2.0, 0.5, 2.0 ** -6, 2.0 ** -7, 447.0, 1.0625, 126.4, 6.5, 7.49]])
    if prec == Q.PREC_INT8:
        a = np.minimum(a, 200.0)
        rnd = lambda v: np.clip(np.rint(v), -127, 127)  # noqa: E731
    else:
        rnd = Q.round_e4m3
    d = EW.boundary_distance(a, prec)
    fin = np.isfinite(d)
    g = rnd(a[fin])
    assert np.array_equal(rnd(a[fin] + 0.999 * d[fin]), g)
    assert np.array_equal(rnd(np.maximum(a[fin] - 0.999 * d[fin], 0.0)), g)
    # the distance is tight: just past it one side changes code for almost every value
    moved = (rnd(a[fin] + 1.001 * d[fin]) != g) | (rnd(a[fin] - 1.001 * d[fin]) != g)
    assert moved.mean() > 0.99


def test_chain_bound_value_is_the_oracle_chain():
    rng = np.random.default_rng(5)
    m, n, k, r = 60, 50, 40, 8
    Ut = rng.uniform(0.5, 1.5, (m, r)).astype(np.float32)
    Vt = rng.uniform(0.5, 1.5, (r, k)).astype(np.float32)
    Wt = rng.uniform(0.5, 1.5, (r, k)).astype(np.float32)
    Zt = rng.uniform(0.5, 1.5, (n, r)).astype(np.float32)
    for prec in ((1, 1, 1), (0, 0, 0), (1, 1, 3)):
        ref, bound = EW.chain_bound(Ut, Vt, Wt, Zt, prec)
        assert np.array_equal(ref, oracle.lramm.chain(Ut, Vt.T, Wt.T, Zt.T, prec))
        assert np.all(bound >= 0)
    # integer chains are exact on both sides: zero bound
    _, b = EW.chain_bound(Ut, Vt, Wt, Zt, (1, 1, 1))
    assert not np.any(b > 1e-30)


def test_lead_tail_bound_catches_a_wrong_residual_scale():
    """A residual term formed with its scale doubled (a plausible slip) lies
    far outside the element-wise bound; the correct FP32 sum of the terms
    lies inside it."""
    MX = oracle.mixed
    rng = np.random.default_rng(9)
    m, n, k, r, lead = 80, 70, 64, 24, 8
    Ut = (rng.standard_normal((m, r)) * np.exp(-np.arange(r) / 8.0)).astype(np.float32)
    Vt = (rng.standard_normal((r, k)) / np.sqrt(k)).astype(np.float32)
    Wt = (rng.standard_normal((r, k)) / np.sqrt(k)).astype(np.float32)
    Zt = (rng.standard_normal((n, r)) * np.exp(-np.arange(r) / 8.0)).astype(np.float32)
    prec = (1, 1, 4)
    ref = MX.chain_lead_tail(Ut, Vt.T, Wt.T, Zt.T, prec, lead, 1, 2)
    bound = EW.lead_tail_bound(Ut, Vt, Wt, Zt, prec, lead, 1, 2)
    E1 = Q.qm(Vt, Wt.T, 1)
    E2 = Q.qm(E1, Zt.T, 1)
    (uh, suh), (ul, sul) = MX.quantize_hilo(Ut[:, :lead], 1, 1)
    (eh, seh), (el, sel) = MX.quantize_hilo(E2[:lead, :], 1, 0)
    terms = [MX._qm_codes(uh, suh, eh, seh, 1, 0), MX._qm_codes(ul, sul, eh, seh, 1, 0),
             MX._qm_codes(uh, suh, el, sel, 1, 0), MX.qm_mxfp4(Ut[:, lead:], E2[lead:, :])]
    fp32_sum = terms[0]
    for t in terms[1:]:
        fp32_sum = (fp32_sum + t).astype(np.float32)
    assert np.all(np.abs(fp32_sum.astype(np.float64) - ref) <= bound)
    wrong = terms[0].astype(np.float64) + 2.0 * terms[1] + terms[2] + terms[3]
    assert np.mean(np.abs(wrong - ref) > bound) > 0.5
