"""CPU oracle for the LRAMM hot path (FP64, plain numpy).

TEST INFRASTRUCTURE.  This package exists to check the CUDA library, not to
run the method: only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import it.  It shares no code with the CUDA
path (paper_2405_16917_gb300/) and never imports it.

Modules:
  philox  -- Philox4x32-10 words and the Gaussian test matrix Omega
  quant   -- symmetric quantiser (Eqs. Quantization, get_lambda,
             Dequantization), e4m3 rounding, QM (Algorithm 2)
  lramm   -- randomized SVD (Sec. 2.2, Algorithm 1, power iterations) and
             LRAMM (Algorithm 3), exact product, relative Frobenius error
  rf      -- the range-finder form C ~ (X Q)(Q^T W) and its gradients
  mixed   -- MXFP4 (e2m1, 32-element block scales), split-precision
             residuals and the lead / tail E3 of the mixed 4/8-bit chain
  qsvd    -- the quantised SVD approximation of one matrix (Algorithm 4)
  sketch8 -- the range finder with its products on e4m3 codes
  tune    -- the probe error estimate and the selection rule of parameter tuning
"""
from . import philox, quant, lramm, rf, mixed, qsvd, sketch8, tune  # noqa: F401
