"""The CPU oracle against facts outside itself (CPU only, no GPU)."""
import numpy as np
import pytest

import oracle
import workloads
from tests import pins


def test_philox_matches_curand_host_generator():
    try:
        n = pins.pin_philox_curand(oracle.philox)
    except RuntimeError as e:
        pytest.skip(str(e))
    assert n > 0


def test_gaussian_statistics():
    pins.pin_gaussian_stats(oracle.philox)


def test_box_muller_closed_forms():
    pins.pin_box_muller_special(oracle.philox)


def test_gaussian_layout():
    """Element e of Omega is output e mod 4 of block e // 4 (word pairs
    (0,1) and (2,3) through Box-Muller), independent of the matrix shape."""
    a = oracle.philox.gaussian_matrix(99, 3, 7, 13).ravel()
    b = oracle.philox.gaussian_matrix(99, 3, 13, 7).ravel()
    assert np.array_equal(a, b)
    w = oracle.philox.philox_words(99, 3, 1, first_block=5)[0]
    z0, z1 = oracle.philox.box_muller(w[0:1], w[1:2])
    z2, z3 = oracle.philox.box_muller(w[2:3], w[3:4])
    assert np.array_equal(a[20:24], np.array([z0[0], z1[0], z2[0], z3[0]], dtype=np.float32))


def test_quantiser_worked_examples():
    pins.pin_quant_golden(oracle.quant)


def test_e4m3_rounding():
    pins.pin_e4m3(oracle.quant)


def test_quantiser_bounds_and_symmetry():
    pins.pin_quant_bounds(oracle.quant)


def test_qm_bruteforce_and_scales():
    pins.pin_qm_bruteforce(oracle.quant)


def test_qm_error_bound():
    pins.pin_qm_error_bound(oracle.quant)


def test_orth_is_unique_thin_qr():
    pins.pin_orth(oracle.lramm)


def test_rsvd_exact_rank():
    pins.pin_rsvd_exact_rank(oracle.lramm, workloads)


def test_rsvd_full_sketch_is_exact_svd():
    pins.pin_rsvd_full_sketch(oracle.lramm)


def test_rsvd_error_bounds():
    pins.pin_rsvd_bounds(oracle.lramm, workloads)


def test_lramm_exact_rank_and_alpha_beta():
    pins.pin_lramm_exact(oracle.lramm, workloads, oracle.quant)


def test_lramm_factor_identity():
    pins.pin_lramm_factor_identity(oracle.lramm, workloads, oracle.quant)


def test_lramm_bit_width_ordering():
    pins.pin_lramm_bit_ordering(oracle.lramm, workloads, oracle.quant)


# ---------------------------------------------------------------- range-finder form
def test_rf_qr_adjoint_matches_finite_differences():
    pins.pin_qr_adjoint_fd(oracle.rf)


def test_rf_gradients_match_finite_differences():
    pins.pin_rf_gradients_fd(oracle.rf)


def test_rf_exact_rank_product():
    pins.pin_rf_exact_rank(oracle.rf)


def test_rf_copyltu():
    pins.pin_copyltu(oracle.rf)


# ---------------------------------------------------------------- MXFP4, residuals, lead / tail
def test_e2m1_grid_and_rounding():
    pins.pin_e2m1(oracle.mixed)


def test_mx_scale_rule():
    pins.pin_mx_scale_rule(oracle.mixed)


def test_mxfp4_quantiser():
    pins.pin_mxfp4_quantise(oracle.mixed)


def test_mx_product_bruteforce():
    pins.pin_mx_product_bruteforce(oracle.mixed)


def test_hilo_residual():
    pins.pin_hilo_residual(oracle.mixed, oracle.quant)


def test_lead_tail_e3():
    pins.pin_lead_tail(oracle.mixed, oracle.quant)


def test_lramm_zero_operand_gives_zero():
    """Degenerate input: LRAMM of a zero operand is exactly zero in every precision."""
    rng = np.random.default_rng(5)
    A = np.zeros((40, 30), dtype=np.float32)
    B = rng.standard_normal((30, 36)).astype(np.float32)
    for prec in ((0, 0, 0), (1, 1, 1), (2, 2, 2), (3, 3, 3)):
        assert np.all(oracle.lramm.lramm(A, B, 6, 2, 1, 7, prec) == 0)
        assert np.all(oracle.lramm.lramm(B.T.copy(), A.T.copy(), 6, 2, 1, 7, prec) == 0)


# Algorithm 4 / Theorem 4.4
def test_qsvd_unquantised():
    pins.pin_qsvd_unquantised(oracle.qsvd, oracle.lramm, workloads, oracle.quant)


def test_qsvd_codes_bruteforce():
    pins.pin_qsvd_codes_bruteforce(oracle.qsvd, oracle.quant)


def test_qsvd_error_bounds():
    pins.pin_qsvd_error_bounds(oracle.qsvd, workloads, oracle.quant)


# E4M3 range finder
def test_rf_e4m3_structure():
    pins.pin_rf_e4m3_structure(oracle.sketch8, oracle.lramm, workloads)


def test_rf_e4m3_product():
    pins.pin_rf_e4m3_product(oracle.sketch8, oracle.quant)


def test_rf_e4m3_accuracy():
    pins.pin_rf_e4m3_accuracy(oracle.sketch8, oracle.lramm, workloads)


# Parameter tuning
def test_probe_error():
    pins.pin_probe_error(oracle.tune)


def test_select():
    pins.pin_select(oracle.tune)
