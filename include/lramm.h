/*
 * lramm.h -- C ABI of the GB300 (sm_103a) LRAMM library.
 *
 * LRAMM (arXiv 2405.16917) approximates C = A B by a randomized SVD of each
 * operand followed by a chain of three quantised factor GEMMs:
 *
 *   RSVD(A, r) = U_r Sigma_r V_r^T,  RSVD(B, r) = W_r Gamma_r Z_r^T
 *   U~ = U_r Sigma_r,  Z~ = Gamma_r Z_r^T                      (Sec. 3.2)
 *   E1 = QM(V_r^T W_r, d1), E2 = QM(E1 Z~, d2), E3 = QM(U~ E2, d3)
 *   D  = alpha E3 + beta C                                     (Algorithm 3)
 *
 * QM is the quantised GEMM of Algorithm 2 with the symmetric linear
 * quantiser of Eqs. (Quantization), (get_lambda), (Dequantization).  The
 * RSVD is the two-stage randomized scheme of Sec. 2.2 (Gaussian sketch with
 * oversampling p, q power iterations) followed by Algorithm 1.
 *
 * Conventions for every entry point:
 *   - Matrices are row-major with a leading dimension (row stride) in
 *     elements.  Device pointers unless stated otherwise.
 *   - `stream` is a cudaStream_t passed as void*.  All device work is
 *     enqueued on it; no entry point synchronises except lramm_status_read.
 *   - The caller owns every device buffer (inputs, outputs, workspace) and
 *     the stream.  A plan owns host metadata only; no entry point other than
 *     lramm_plan_create/destroy allocates or frees host memory, and none
 *     allocates device memory.
 *   - Argument errors are returned synchronously and nothing is enqueued.
 *     Errors found on the device (Cholesky breakdown, Jacobi not converged)
 *     are latched in a status word at the start of the workspace and
 *     returned by lramm_status_read.  Nothing throws across the ABI.
 *   - On any error the contents of output buffers are unspecified.
 */
#ifndef LRAMM_H
#define LRAMM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LRAMM_API __attribute__((visibility("default")))
#else
#define LRAMM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LRAMM_OK = 0,
  LRAMM_ERR_INVALID_ARG = 1,   /* bad shape, stride, pointer or option        */
  LRAMM_ERR_UNSUPPORTED = 2,   /* valid but not implemented (e.g. l > 576)    */
  LRAMM_ERR_WORKSPACE = 3,     /* workspace smaller than lramm_workspace_size */
  LRAMM_ERR_CUDA = 4,          /* a CUDA runtime call failed                  */
  LRAMM_ERR_NUMERIC = 5,       /* Cholesky pivot <= 0 in an orthonormalisation */
  LRAMM_ERR_TIMEOUT = 6,       /* a bounded device wait ran out               */
  LRAMM_WARN_NOCONV = 7        /* Jacobi SVD hit its sweep cap                */
} lramm_status;

/* Storage type of the operands A and B. */
typedef enum { LRAMM_F32 = 0, LRAMM_BF16 = 1 } lramm_dtype;

/* Precision d_i of each QM in Algorithm 3.
 *   F32  : no quantisation, FP32 product (the "plain LRAMM" of Sec. 4.2)
 *   INT8 : N = 8 bits, codes in [-127, 127], exact integer product
 *   INT4 : N = 4 bits, codes in [-7, 7], exact integer product
 *   E4M3 : FP8 e4m3 codes with lambda = 448 / a_max, FP32 accumulation
 *   MXFP4: e2m1 elements, one power-of-two scale 2^e per 32 consecutive
 *          elements along K, e = ceil(log2(a_max / 6)) (OCP MX e2m1 with this
 *          scale rule); exact block sums, FP32 sum over blocks.  The scale
 *          groups of lramm_scale do not apply to MXFP4 operands.          */
typedef enum { LRAMM_P_F32 = 0, LRAMM_P_INT8 = 1, LRAMM_P_INT4 = 2, LRAMM_P_E4M3 = 3, LRAMM_P_MXFP4 = 4 } lramm_prec;

/* Scale groups of the quantiser (a_max of Eq. (get_lambda)):
 *   ROWCOL: left operand one scale per row, right operand one per column
 *   TENSOR: one scale per operand (the paper's per-matrix a_max)          */
typedef enum { LRAMM_S_ROWCOL = 0, LRAMM_S_TENSOR = 1 } lramm_scale;

/* Arithmetic of the products that touch A or B (sketch, power iterations,
 * projection); the orthonormalisations and small SVD are FP32.
 *   F32  : FP32-accurate products
 *   TF32 : one TF32 pass (10-bit mantissa operands), FP32 accumulate
 *   BF16 : BF16 operands, FP32 accumulate
 *   E4M3 : the range finder of the SVD form (the sketch X Omega and the
 *          power iterations) on FP8 e4m3 codes, FP32 accumulate: X is
 *          quantised once per call per row (for X B) and per column (for
 *          X^T B), each l-column matrix B per column, products dequantised
 *          as in Algorithm 2; the projection B^T = X^T Q stays TF32.  FP32
 *          operands only (else LRAMM_ERR_UNSUPPORTED at plan creation);
 *          the range-finder form rejects it (LRAMM_ERR_UNSUPPORTED).     */
typedef enum {
  LRAMM_SKETCH_F32 = 0,
  LRAMM_SKETCH_TF32 = 1,
  LRAMM_SKETCH_BF16 = 2,
  LRAMM_SKETCH_E4M3 = 3
} lramm_sketch;

typedef struct lramm_desc {
  int64_t m, n, k;        /* A is m x k, B is k x n, C and D are m x n           */
  int64_t lda, ldb, ldc;  /* row strides of A, B and of C / D (elements)         */
  int32_t a_type, b_type; /* lramm_dtype of A and B                              */
  int32_t r;              /* target rank, 1 <= r                                 */
  int32_t p;              /* oversampling: l = r + p sketch columns, l <= 576
                             (the SVD form: l <= 544, the small SVD's limit),
                             l <= min(m, k) and l <= min(k, n)                   */
  int32_t q;              /* power iterations, 0 <= q <= 16                      */
  uint64_t seed;          /* Philox4x32-10 key; Omega_A is stream 0, Omega_B 1   */
  int32_t prec[3];        /* lramm_prec of E1, E2, E3 (d1, d2, d3)               */
  int32_t scale;          /* lramm_scale                                         */
  int32_t sketch;         /* lramm_sketch                                        */
  float alpha, beta;      /* D = alpha E3 + beta C                               */
  int32_t max_sweeps;     /* Jacobi sweep cap, 0 selects the default (40)        */
  int32_t flags;          /* LRAMM_FLAG_* bits; other bits must be 0             */
  /* Mixed precision inside E3 = QM(U~ E2): the first `lead` rank directions
   * (the largest singular values) in lead_prec (INT8, INT4 or E4M3), the
   * remaining r - lead in prec[2]:
   *   E3 = QM(U~_l^hi, E2_l^hi) [+ QM(U~_l^lo, E2_l^hi)] [+ QM(U~_l^hi, E2_l^lo)]
   *        + QM(U~_t, E2_t)
   * where x^lo is the quantised residual x - deq(x^hi) (its own scales);
   * lead_split = 0, 1 or 2 selects the bracketed terms in order.  lead = 0
   * disables the split (lead_prec and lead_split are then ignored). */
  int32_t lead;
  int32_t lead_prec;
  int32_t lead_split;
} lramm_desc;

/* flags: record a CUDA event pair around every kernel launch of a call, on
 * the call's stream, so lramm_timing_read can attribute device time per
 * kernel kind (the per-operator time split of Sec. 4.1, Fig. 2). */
#define LRAMM_FLAG_TIMING 1
/* flags: lramm_matmul records its ~110 launches once into a CUDA graph (stream
 * capture on the call's stream) and replays the graph on later calls with the
 * same A, B, C, D, workspace, stream and device; any other arguments capture
 * a new graph.  Ignored with LRAMM_FLAG_TIMING or on the legacy default
 * stream (0), which cannot be captured.  The caller keeps the captured
 * buffers alive while the plan may replay them. */
#define LRAMM_FLAG_GRAPH 2
/* flags, for tests of the failure path: every bounded device wait of the
 * small SVD's thread-block cluster (the block moves of the cluster Jacobi)
 * gives up after about 2^20 SM clock cycles (half a millisecond) instead of
 * about 2^30 (half a second). */
#define LRAMM_FLAG_SHORT_WAITS 4
/* flags, for tests of the failure path: one CTA of the cluster Jacobi (rank
 * 1, in clusters of two or more CTAs) skips its first block move, so that
 * its neighbours' bounded waits expire.  The call then latches
 * LRAMM_ERR_TIMEOUT in the status word, every CTA waits (bounded) for the
 * copies already issued into it, the launch returns and the context stays
 * usable; the call's outputs are undefined. */
#define LRAMM_FLAG_TEST_DROP_MOVE 8

/* Kernel kinds reported by lramm_timing_read. */
typedef enum {
  LRAMM_K_OMEGA = 0,      /* Philox Gaussian test matrix                      */
  LRAMM_K_SKETCH = 1,     /* products with A or B (sketch, power, projection) */
  LRAMM_K_GRAM = 2,       /* Gram matrices of CholeskyQR                      */
  LRAMM_K_CHOL = 3,       /* l x l Cholesky                                   */
  LRAMM_K_TRSM = 4,       /* Q = Y L^-T                                       */
  LRAMM_K_RFACTOR = 5,    /* R = R2 R1; in quantised chains also the l x r    */
                          /* factor R1 U_s Sigma^-1 of the right factors      */
  LRAMM_K_SVD = 6,        /* one-sided Jacobi SVD of R^T                      */
  LRAMM_K_SVDSORT = 7,    /* sort / truncate to rank r                        */
  LRAMM_K_ASSEMBLE = 8,   /* U~, V^T, W^T, Z~^T from the small SVD            */
  LRAMM_K_QUANT = 9,      /* absmax + quantise of a QM operand                */
  LRAMM_K_E1 = 10,        /* QM E1                                            */
  LRAMM_K_E2 = 11,        /* QM E2                                            */
  LRAMM_K_E3 = 12,        /* QM E3 with the alpha/beta epilogue               */
  LRAMM_K_OTHER = 13,
  LRAMM_K_BWD = 14,       /* range-finder backward: products with G, X, W, Q  */
  LRAMM_K_ADJOINT = 15,   /* range-finder backward: thin-QR adjoints          */
  LRAMM_K_RECON = 16,     /* Algorithm 4: code conversion + product U~' V'^T  */
  LRAMM_K_COUNT = 17
} lramm_kernel_kind;

typedef struct lramm_plan_s* lramm_plan_t;

/* Validate a problem description and build a plan (host metadata only).
 * Returns LRAMM_ERR_INVALID_ARG for inconsistent sizes or options,
 * LRAMM_ERR_UNSUPPORTED for l = r + p > 576 (the orthonormalisation's
 * limit).  The SVD form (lramm_rsvd, lramm_matmul, lramm_qsvd) also needs
 * the small SVD to fit, l <= 544; those calls return LRAMM_ERR_UNSUPPORTED
 * beyond it, the range-finder form runs to 576.  *out is set only on
 * success. */
LRAMM_API lramm_status lramm_plan_create(const lramm_desc* desc, lramm_plan_t* out);

/* Release a plan.  NULL is accepted. */
LRAMM_API lramm_status lramm_plan_destroy(lramm_plan_t plan);

/* Bytes of device workspace lramm_matmul / lramm_rsvd / lramm_chain need.
 * The workspace must be 256-byte aligned; its first 256 bytes hold the
 * device status word. */
LRAMM_API lramm_status lramm_workspace_size(lramm_plan_t plan, size_t* bytes);

/* Randomized SVD of one operand (Sec. 2.2 range finder with q power
 * iterations, then Algorithm 1), truncated to rank r.
 *   which = 0: X is A (m x k, stride lda, type a_type), Omega stream 0
 *   which = 1: X is B (k x n, stride ldb, type b_type), Omega stream 1
 * Outputs (device, FP32, row-major, dense): U rows x r, S r (descending),
 * V cols x r, with X ~ U diag(S) V^T.  The sign of each (U_i, V_i) pair is
 * not canonicalised. */
LRAMM_API lramm_status lramm_rsvd(lramm_plan_t plan, int32_t which, const void* X,
                        float* U, float* S, float* V,
                        void* ws, size_t ws_bytes, void* stream);

/* LRAMM, Algorithm 3: D = alpha * E3 + beta * C (m x n, FP32, stride ldc).
 * A and B as described by the plan.  C may be NULL when beta == 0 and may
 * alias D. */
LRAMM_API lramm_status lramm_matmul(lramm_plan_t plan, const void* A, const void* B,
                          const float* C, float* D,
                          void* ws, size_t ws_bytes, void* stream);

/* The quantised factor chain of Algorithm 3 on given factors (all FP32,
 * row-major, dense):
 *   Ut  m x r : U~ = U_r Sigma_r           Vt r x k : V_r^T
 *   Wt  r x k : W_r^T                      Zt n x r : Z~^T = Z_r Gamma_r
 * computes E1 = QM(Vt Wt^T, d1), E2 = QM(E1 Zt^T, d2), E3 = QM(Ut E2, d3),
 * D = alpha E3 + beta C (stride ldc). */
LRAMM_API lramm_status lramm_chain(lramm_plan_t plan, const float* Ut, const float* Vt,
                         const float* Wt, const float* Zt, const float* C, float* D,
                         void* ws, size_t ws_bytes, void* stream);

/* Wait for `stream`, read and clear the status word at the start of `ws`.
 * Returns the first device error latched since the last read, or LRAMM_OK. */
LRAMM_API lramm_status lramm_status_read(const void* ws, void* stream);

/* Wait for `stream` and copy the first n (1..64) 32-bit words of the
 * workspace's status area into info (host): info[0] = the status word,
 * info[1], info[2] = Jacobi sweeps of the A- and B-side SVDs of the last
 * call, info[3] bit 0 = the last lramm_matmul assembled its factors with
 * TF32 tensor-core products (quantised chains in a tensor-core sketch mode),
 * else with FP32 products; info[20], info[21] = how many Cholesky
 * factorisations of the A- and B-side randomized SVDs met a non-positive
 * pivot and took the shifted CholeskyQR fallback (larger shift, then a third
 * pass where the orthonormalisation had two).  Nothing is cleared. */
LRAMM_API lramm_status lramm_info_read(const void* ws, int32_t* info, int32_t n, void* stream);

/* Static description of a status code. */
LRAMM_API const char* lramm_status_str(lramm_status s);

/* Source location and CUDA error name/string of the last CUDA runtime call
 * that failed in this thread (LRAMM_ERR_CUDA), or "" if none did. */
LRAMM_API const char* lramm_last_cuda_error(void);

/* Device time of the most recent lramm_matmul / lramm_rsvd / lramm_chain
 * call of a plan created with LRAMM_FLAG_TIMING, per lramm_kernel_kind:
 * ms[kind] = summed event time, launches[kind] = number of launches (arrays
 * of LRAMM_K_COUNT entries, host memory).  Waits for the recorded events.
 * Returns LRAMM_ERR_INVALID_ARG when the plan was created without the flag. */
LRAMM_API lramm_status lramm_timing_read(lramm_plan_t plan, float* ms, int32_t* launches);

/* Static name of a kernel kind ("sketch", "e3", ...). */
LRAMM_API const char* lramm_kernel_kind_name(int32_t kind);

/* ---- building blocks, exposed for parity tests -------------------------- */

/* Philox4x32-10 words of blocks 0 .. n_blocks-1 (counter (n, 0, stream_id, 0),
 * key (lo32 seed, hi32 seed)); out is n_blocks x 4 uint32 (device). */
LRAMM_API lramm_status lramm_philox_words(uint64_t seed, uint32_t stream_id, int64_t n_blocks,
                                uint32_t* out, void* stream);

/* The Gaussian test matrix Omega (rows x cols, FP32, row-major, dense):
 * element e = i * cols + j is Box-Muller output e mod 4 of Philox block
 * e / 4 (Sec. 2.2, Gaussian sampling). */
LRAMM_API lramm_status lramm_gaussian(uint64_t seed, uint32_t stream_id, int64_t rows, int64_t cols,
                            float* out, void* stream);

/* Symmetric quantiser, Eqs. (get_lambda) and (Quantization), per row
 * (per_row = 1) or per tensor (per_row = 0) of X (rows x cols, stride ldx):
 * lambda = D / a_max in FP32, code = rint(x * lambda) clamped to +-D
 * (INT8: D = 127, INT4: D = 7) or rounded to e4m3 (E4M3: D = 448).
 * codes: rows x ldcodes; INT8 codes are stored as bfloat16 values, INT4 and
 * E4M3 codes as e4m3 bytes; columns cols .. ldcodes-1 are set to zero.
 * scales: one FP32 dequantisation scale a_max / D per row (per_row = 1) or
 * one value (per_row = 0).  Needs ws of lramm_quant_ws_bytes() bytes for
 * per-tensor mode (may be NULL for per-row mode). */
LRAMM_API lramm_status lramm_quantize(const float* X, int64_t rows, int64_t cols, int64_t ldx,
                            int32_t prec, int32_t per_row, void* codes, int64_t ldcodes,
                            float* scales, void* ws, void* stream);

/* Per-column symmetric quantiser (Eqs. get_lambda, Quantization, one scale
 * per column of X): the columns of X (rows x cols, stride ldx, FP32) become
 * the rows of a K-major code matrix codesT (cols x ldcodes, ldcodes >= rows,
 * zero beyond rows), codes as lramm_quantize writes them for prec;
 * scales[cols] = a_max / D.  The same decisions as lramm_quantize applied to
 * X^T.  ws: device scratch of cols 32-bit words.  Asynchronous on `stream`. */
LRAMM_API lramm_status lramm_quantize_cols(const float* X, int64_t rows, int64_t cols, int64_t ldx, int32_t prec,
                                           void* codesT, int64_t ldcodes, float* scales, void* ws, void* stream);

/* QM product of Algorithm 2 on quantised codes, both K-major:
 *   L  M x K (stride ldl), Rt N x K (stride ldr); codes as lramm_quantize
 *   writes them for `prec`.  acc(i,j) = sum_t L(i,t) Rt(j,t), exact for
 *   INT8/INT4, FP32-accumulated for E4M3.
 *   out_kind 0: D(i,j) = alpha * fp32(acc) * (sL[i or 0] * sR[j or 0])
 *                        + beta * C(i,j)           (FP32, stride ldd)
 *   out_kind 1: D receives acc itself, int32 for INT8/INT4, FP32 for E4M3.
 * per_row = 1: sL, sR have M and N entries; 0: one entry each.
 * K must be a multiple of 16; C may be NULL when beta == 0. */
LRAMM_API lramm_status lramm_qgemm(const void* L, const void* Rt, int64_t M, int64_t N, int64_t K,
                         int64_t ldl, int64_t ldr, int32_t prec, int32_t per_row,
                         const float* sL, const float* sR, float alpha, float beta,
                         const float* C, int64_t ldc, void* D, int64_t ldd,
                         int32_t out_kind, void* stream);

/* Range-finder form of LRAMM as a linear layer: the two-stage randomized
 * scheme of Sec. 2.2 applied to the right operand.  C ~ X W is computed as
 * (X Q)(Q^T W): Q (k x l, l = r + p) is the orthonormal basis of the sketch
 * W Omega (Omega n x l, Philox stream 1 of the plan's seed) after q power
 * iterations (text after Eq. (rsvderror_z)), every product re-orthonormalised
 * by CholeskyQR; T = X Q (m x l), P = Q^T W (l x n), and
 *   C = alpha * QM(T P, d) + beta * C      (Algorithm 2, d = prec[2], plan scale)
 * or alpha T P + beta C when prec[2] is LRAMM_P_F32.  X: m x k of a_type,
 * stride lda; W: k x n of b_type, stride ldb; C: m x n FP32, stride ldc, read
 * when beta != 0 and written.  The plan's r, p, q, seed, prec[2], scale,
 * sketch, alpha and beta apply; ws as for lramm_matmul.  Asynchronous on
 * `stream`; device-side errors latch in the status word. */
LRAMM_API lramm_status lramm_rf_forward(lramm_plan_t plan, const void* X, const void* W, float* C, void* ws,
                                        size_t ws_bytes, void* stream);

/* Gradients of L = <G, C> for the range-finder form, with Omega fixed and the
 * quantiser passed straight through (the gradients of alpha X Q Q^T W):
 *   dT = alpha G P^T, dP = alpha T^T G, dX = dT Q^T, dW = Q dP + the path
 *   through Q: dQ = X^T dT + W dP^T carried back through every thin QR
 *   Y = Q R by dY = (dQ + Q copyltu(M)) R^-T, M = -dQ^T Q, and through every
 *   product of the power chain (W Z: dW += dY Z^T; W^T Q: dW += Q dY^T; the
 *   sketch W Omega: dW += dY Omega^T).
 * The range finder is recomputed (no state is kept from lramm_rf_forward).
 * G: m x n FP32 (stride ldc); dX: m x k FP32 (dense, stride k); dW: k x n
 * FP32 (dense, stride n).  W must be FP32 (else LRAMM_ERR_UNSUPPORTED).  ws as
 * for lramm_matmul. */
LRAMM_API lramm_status lramm_rf_backward(lramm_plan_t plan, const void* X, const void* W, const float* G,
                                         float* dX, float* dW, void* ws, size_t ws_bytes, void* stream);

/* The QM product of Algorithm 2 on the tensor cores, on the codes
 * lramm_quantize writes:
 *   prec LRAMM_P_INT8: codes as bfloat16 values (exact BF16 operands),
 *     tcgen05.mma kind::f16; each CTA adds at most 1024 products in FP32,
 *     where every partial sum is an exact integer; longer K is split across
 *     CTAs and the partials are added as 32-bit integers: exact.
 *   prec LRAMM_P_INT4: codes as FP8 e4m3 bytes (|c| <= 7 are exact e4m3
 *     values), kind::f8f6f4; FP32 sums of products <= 49: exact for
 *     K < 342000 (larger K: LRAMM_ERR_UNSUPPORTED).
 *   prec LRAMM_P_E4M3: e4m3 codes, kind::f8f6f4; FP32 sums.
 *   acc(i,j) = sum_t L(i,t) Rt(j,t), L M x K (stride ldl), Rt N x K (stride ldr), then
 *   D(i,j) = alpha * fp32( fp32(acc) * fp32(sL[i or 0] * sR[j or 0]) ) + beta * C(i,j)
 * (FP32, stride ldd), as lramm_qgemm with out_kind 0.  per_row as in
 * lramm_qgemm.  K a multiple of 16; L and Rt 16-byte aligned with row
 * pitches (ldl, ldr times the code size) multiples of 16 bytes (else
 * LRAMM_ERR_UNSUPPORTED).  ws: device buffer of
 * lramm_qgemm_tc_ws_bytes(prec, M, N, K) bytes, 256-byte aligned (first
 * word: the status word, LRAMM_ERR_TIMEOUT if a bounded wait expired; then
 * the split-K partials).  Asynchronous on `stream`. */
LRAMM_API lramm_status lramm_qgemm_tc(int32_t prec, const void* L, const void* Rt, int64_t M, int64_t N, int64_t K,
                                      int64_t ldl, int64_t ldr, int32_t per_row, const float* sL,
                                      const float* sR, float alpha, float beta, const float* C, int64_t ldc,
                                      float* D, int64_t ldd, void* ws, size_t ws_bytes, void* stream);

/* Bytes of workspace lramm_qgemm_tc needs for an M x N x K product. */
LRAMM_API size_t lramm_qgemm_tc_ws_bytes(int32_t prec, int64_t M, int64_t N, int64_t K);

/* C = alpha A B^T + beta C on the tensor cores with FP32 operands rounded
 * to TF32 (tcgen05.mma kind::tf32, FP32 accumulation): the dense products
 * with the l-column factors of the range-finder backward (dX = dT Q^T,
 * dW = Q dP + ...).  A: M x K (stride lda), B: N x K (stride ldb), C: M x N
 * (stride ldc), all FP32 row-major, C updated in place.  A and B 16-byte
 * aligned, lda and ldb multiples of 4 (else LRAMM_ERR_UNSUPPORTED).  ws:
 * lramm_tgemm_tc_ws_bytes(M, N, K) bytes, 256-byte aligned (status word,
 * then split-K partials).  Asynchronous on `stream`. */
LRAMM_API lramm_status lramm_tgemm_tc(int64_t M, int64_t N, int64_t K, float alpha, const float* A, int64_t lda,
                                      const float* B, int64_t ldb, float beta, float* C, int64_t ldc, void* ws,
                                      size_t ws_bytes, void* stream);
LRAMM_API size_t lramm_tgemm_tc_ws_bytes(int64_t M, int64_t N, int64_t K);

/* The products of an operand with an l-column matrix that the range finder
 * runs (Sec. 2.2 sketch Y = X Omega, the power-iteration products, and the
 * projection B^T = X^T Q of Algorithm 1):
 *   transpose = 0: out = X B    (X rows x cols, B cols x l, out rows x l)
 *   transpose = 1: out = X^T B  (B rows x l, out cols x l)
 * X has row stride ldx and type x_type; B and out are dense row-major FP32.
 * sketch = LRAMM_SKETCH_F32: FP32 SIMT product (compensated accumulation).
 * LRAMM_SKETCH_TF32 / LRAMM_SKETCH_BF16, tcgen05 tensor cores, FP32
 * accumulation:
 *   FP32 X: TF32 inputs (kind::tf32; l and ldx divisible by 4, l <= 512);
 *   BF16 X: X exact (kind::f16), B split into BF16 parts B_hi + B_lo (TF32
 *     mode, 16 significant bits of B) or rounded to B_hi (BF16 mode); l
 *     divisible by 4, ldx by 8, any l (blocks of <= 512 columns).
 * X and B 16-byte aligned, else LRAMM_ERR_UNSUPPORTED.  ws:
 * lramm_sketch_ws_bytes(rows, cols, l) bytes, 256-byte aligned (status word,
 * split-K partials, the BF16 parts of B). */
LRAMM_API lramm_status lramm_sketch_product(const void* X, int64_t rows, int64_t cols, int64_t ldx,
                                            int32_t x_type, int32_t transpose, const float* B, int64_t l,
                                            float* out, int32_t sketch, void* ws, size_t ws_bytes,
                                            void* stream);

/* Direct quantised product D = alpha QM(A B, prec) + beta C (Algorithm 2 on
 * the full operands: the paper's DQ8 / DQ4 comparators of Sec. 4.2).  A: m x k
 * (stride lda), B: k x n (stride ldb), FP32 row-major; A is quantised per
 * row and B per column (LRAMM_S_ROWCOL) or each per tensor (LRAMM_S_TENSOR),
 * with the decisions and dequantisation of lramm_quantize / lramm_qgemm;
 * prec INT8, INT4 or E4M3 (exact integer sums for INT8 / INT4).  ws:
 * lramm_dq_ws_bytes(prec, m, n, k) bytes, 256-byte aligned (status word,
 * codes, scales, split-K partials).  Asynchronous on `stream`. */
LRAMM_API lramm_status lramm_dq_matmul(int32_t prec, int32_t scale, int64_t m, int64_t n, int64_t k, float alpha,
                                       const float* A, int64_t lda, const float* B, int64_t ldb, float beta,
                                       const float* C, int64_t ldc, float* D, int64_t ldd, void* ws, size_t ws_bytes,
                                       void* stream);
LRAMM_API size_t lramm_dq_ws_bytes(int32_t prec, int64_t m, int64_t n, int64_t k);

/* Number of CUDA kernels the library has launched in this process so far
 * (all plans and threads): the difference around a region counts its launches. */
LRAMM_API uint64_t lramm_launch_count(void);

/* MXFP4 quantiser (lramm_prec LRAMM_P_MXFP4) of the rows of X (rows x cols,
 * stride ldx, FP32): per row and per 32 consecutive elements, e = ceil(log2(
 * fp32(a_max / 6))) clamped to [-127, 127] (-127 for a zero block), element
 * = x 2^-e rounded to nearest-even on the e2m1 grid.  codes: rows x ldcodes
 * int8 holding twice the e2m1 value (integers in [-12, 12]), zero beyond
 * cols; exps: rows x (ldcodes / 32) int8.  ldcodes a multiple of 32,
 * >= cols.  Asynchronous on `stream`. */
LRAMM_API lramm_status lramm_quantize_mx(const float* X, int64_t rows, int64_t cols, int64_t ldx, int8_t* codes,
                                         int64_t ldcodes, int8_t* exps, void* stream);

/* Block-scaled QM product on MXFP4 codes as lramm_quantize_mx writes them:
 *   acc(i,j) = sum_b 2^(eL[i,b] + eR[j,b] - 2) sum_{t in block b} L(i,t) Rt(j,t)
 * (exact block sums, FP32 sum over blocks in block order), D = alpha acc +
 * beta C (FP32, strides ldc, ldd).  L M x K (stride ldl), Rt N x K (stride
 * ldr), exps M x K/32 and N x K/32; K a multiple of 32, ldl and ldr
 * multiples of 16, code bases 16-byte aligned. */
LRAMM_API lramm_status lramm_qgemm_mx(const int8_t* L, const int8_t* Le, const int8_t* Rt, const int8_t* Re,
                                      int64_t M, int64_t N, int64_t K, int64_t ldl, int64_t ldr, float alpha,
                                      float beta, const float* C, int64_t ldc, float* D, int64_t ldd, void* stream);

/* Quantised SVD approximation of one operand, Algorithm 4 (its error is
 * bounded by Theorem 4.4): the randomized SVD of lramm_rsvd truncated to
 * rank r, U~ = U_r Sigma_r (rows x r) and V_r (cols x r), each quantised by
 * rows along the rank index with Eqs. (get_lambda) and (Quantization): U~
 * with d1 = prec_u, V_r with d2 = prec_v; one scale per row (plan scale
 * LRAMM_S_ROWCOL) or one per factor (LRAMM_S_TENSOR).
 *   which   0: X is the plan's A (rows m, cols k, stride lda, type a_type),
 *           1: its B (rows k, cols n); the sketch as lramm_rsvd draws it.
 *   prec_u, prec_v   LRAMM_P_INT8, LRAMM_P_INT4 or LRAMM_P_E4M3
 *           (LRAMM_P_MXFP4: LRAMM_ERR_UNSUPPORTED).
 *   Uc, Us  codes of U~, rows x ldq, in the format lramm_quantize writes for
 *           prec_u (INT8 as bfloat16 values, INT4 / E4M3 as e4m3 bytes),
 *           columns r .. ldq-1 zero; FP32 scales a_max / D, rows entries or
 *           one.  Vc, Vs: the same for V_r (cols x ldq, prec_v).
 *   ldq     a multiple of 32, >= r; Uc and Vc 16-byte aligned.
 *   Uf, Vf  optional (NULL to skip): the FP32 factors that were quantised,
 *           U~ rows x r and V_r cols x r, row-major, dense.
 *   Xr      optional (NULL to skip): the approximation deq(U~') deq(V')^T,
 *           rows x cols FP32 with stride ldxr >= cols:
 *             Xr(i,j) = fp32(acc) * fp32(su_i * sv_j),
 *             acc = sum_t cu(i,t) cv(j,t)
 *           exact for INT8 / INT4 codes, FP32-accumulated when E4M3 codes
 *           take part.  The pair INT8 / E4M3 has no common code product:
 *           with it Xr must be NULL (else LRAMM_ERR_UNSUPPORTED).
 *   ws      device workspace of lramm_qsvd_ws_bytes(plan, which, prec_u,
 *           prec_v) bytes, 256-byte aligned; its first word is the status
 *           word of lramm_status_read.
 * All outputs are caller-owned device memory; the call is asynchronous on
 * `stream`.  Arguments are checked before anything is launched. */
LRAMM_API lramm_status lramm_qsvd(lramm_plan_t plan, int32_t which, const void* X, int32_t prec_u,
                                  int32_t prec_v, void* Uc, float* Us, void* Vc, float* Vs, int64_t ldq,
                                  float* Uf, float* Vf, float* Xr, int64_t ldxr, void* ws, size_t ws_bytes,
                                  void* stream);

/* Workspace bytes of lramm_qsvd (the plan's workspace plus the code
 * conversion and split-K buffers of the product); 0 for invalid arguments. */
LRAMM_API size_t lramm_qsvd_ws_bytes(lramm_plan_t plan, int32_t which, int32_t prec_u, int32_t prec_v);

/* Bytes of workspace lramm_sketch_product needs for an l-column product of a
 * rows x cols operand. */
LRAMM_API size_t lramm_sketch_ws_bytes(int64_t rows, int64_t cols, int64_t l);

/* Bytes of workspace lramm_quantize needs in per-tensor mode. */
LRAMM_API size_t lramm_quant_ws_bytes(void);

/* lramm_quantize without the caller-supplied workspace.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory
 * themselves -- for example code running under a framework that owns all
 * GPU memory through its own pool and forbids raw device allocations, or a
 * plug-in whose host gives it no allocator.  Arguments, codes and scales
 * are exactly those of lramm_quantize (the caller still passes X, codes
 * and scales).
 * Scratch: per-tensor mode (per_row = 0) keeps its single 32-bit a_max
 * accumulator in a 256-byte array compiled into the library
 * (lramm_noalloc_scratch_bytes()); every GPU that loads the library holds
 * that array until the process exits.  A call that would need more scratch
 * than the array holds is rejected with LRAMM_ERR_UNSUPPORTED; per-row mode
 * uses no scratch.  Nothing is allocated: no cudaMalloc, no cudaFree.
 * The first per-tensor call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture on the device.
 * All calls share the one array: each call clears the accumulator before
 * using it, but calls whose kernels overlap on the GPU (different streams,
 * no ordering between them) race on it and may produce wrong scales. */
LRAMM_API lramm_status lramm_quantize_noalloc(const float* X, int64_t rows, int64_t cols, int64_t ldx,
                                              int32_t prec, int32_t per_row, void* codes,
                                              int64_t ldcodes, float* scales, void* stream);

/* Size in bytes of the scratch array used by lramm_quantize_noalloc. */
LRAMM_API size_t lramm_noalloc_scratch_bytes(void);

#ifdef __cplusplus
}
#endif
#endif /* LRAMM_H */
