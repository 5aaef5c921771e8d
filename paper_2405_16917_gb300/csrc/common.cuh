// Shared device/host helpers of the LRAMM CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "../../include/lramm.h"

namespace lramm {

// First device error wins; later ones are dropped.
__device__ __forceinline__ void set_status(int* st, int code) {
  if (st) atomicCAS(st, 0, code);
}

__host__ __device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// Code containers of the quantised factors: INT8 codes as bfloat16 values
// (exact: |code| <= 127 < 2^8), INT4 and E4M3 codes as e4m3 bytes (|int4| <= 7
// is exact in e4m3).
enum CodeType : int { CODE_BF16 = 0, CODE_E4M3 = 1 };

__host__ __device__ __forceinline__ int code_type_of(int prec) {
  return prec == LRAMM_P_INT8 ? CODE_BF16 : CODE_E4M3;
}
__host__ __device__ __forceinline__ int code_bytes_of(int prec) { return prec == LRAMM_P_INT8 ? 2 : 1; }
__host__ __device__ __forceinline__ float qmax_of(int prec) {
  return prec == LRAMM_P_INT8 ? 127.0f : (prec == LRAMM_P_INT4 ? 7.0f : 448.0f);
}

__device__ __forceinline__ float e4m3_to_float(uint8_t b) {
  __nv_fp8_e4m3 v;
  v.__x = b;
  return static_cast<float>(v);
}

__device__ __forceinline__ float load_as_float(const float* p) { return *p; }
__device__ __forceinline__ float load_as_float(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// Host-side launch helpers -----------------------------------------------
// The last failing CUDA call of this thread, for lramm_last_cuda_error().
void note_cuda_error(cudaError_t e, const char* where);

#define LRAMM_STR2(x) #x
#define LRAMM_STR(x) LRAMM_STR2(x)
#define LRAMM_CUDA_TRY(expr)                                          \
  do {                                                                \
    cudaError_t _e = (expr);                                          \
    if (_e != cudaSuccess) {                                          \
      ::lramm::note_cuda_error(_e, __FILE__ ":" LRAMM_STR(__LINE__)); \
      return LRAMM_ERR_CUDA;                                          \
    }                                                                 \
  } while (0)

#define LRAMM_TRY(expr)                                       \
  do {                                                        \
    lramm_status _s = (expr);                                 \
    if (_s != LRAMM_OK) return _s;                            \
  } while (0)

// Streaming multiprocessors of the calling thread's current device (queried
// once per device): grids and split-K counts are sized from it.
int num_sms();

// The dynamic shared-memory cap of a kernel (cudaFuncAttributeMax-
// DynamicSharedMemorySize) belongs to the function, not to a launch.  A
// captured CUDA graph's kernel node keeps its own size, but a node that is
// launched again on its own (as a profiler replaying the graph does) is
// checked against the function's current cap -- the last value any launch
// set, possibly a smaller one from another shape.  So the cap is raised
// once per kernel and device to the device's opt-in maximum (less the
// kernel's static shared memory), and only a launch needing more than that
// is refused (cudaErrorInvalidValue).
cudaError_t smem_cap_fn(const void* fn, size_t need);
template <typename F>
inline cudaError_t smem_cap(F* fn, size_t need) {
  return smem_cap_fn(reinterpret_cast<const void*>(fn), need);
}

// Every kernel launch of the library is followed by exactly one check;
// the check also counts the launch (lramm_launch_count).
void count_launch();

inline lramm_status last_launch_at(const char* where) {
  count_launch();
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return LRAMM_OK;
  note_cuda_error(e, where);
  return LRAMM_ERR_CUDA;
}
#define last_launch() ::lramm::last_launch_at(__FILE__ ":" LRAMM_STR(__LINE__))

// ---- kernels implemented in the .cu files (host launchers) ---------------

// philox.cu
lramm_status launch_philox_words(uint64_t seed, uint32_t sid, int64_t n_blocks, uint32_t* out,
                                 cudaStream_t s);
lramm_status launch_gaussian(uint64_t seed, uint32_t sid, int64_t rows, int64_t cols, float* out,
                             int64_t ldo, cudaStream_t s);

// gemm_simt.cu: C = alpha * op(A) op(B) + beta * C, FP32 accumulation.
// op(A) is M x K: ta = 0 -> A[m*lda + k], ta = 1 -> A[k*lda + m].
// op(B) is K x N: tb = 0 -> B[k*ldb + n], tb = 1 -> B[n*ldb + k].
// a_bf16 = 1 reads A as bfloat16 (same layout rules).
// Predicated launches (cond != nullptr): the kernels of this library that
// take a `cond` device word do nothing while it is 0 -- the optional extra
// work of the CholeskyQR fallback is enqueued unconditionally and runs only
// when a breakdown set the word.
lramm_status sgemm(int ta, int tb, int64_t M, int64_t N, int64_t K, float alpha, const void* A,
                   int64_t lda, int a_bf16, const float* B, int64_t ldb, float beta, float* C,
                   int64_t ldc, cudaStream_t s, const int* cond = nullptr);

// smallla.cu -- small dense linear algebra, batched over up to two problems
// (the A-side and B-side randomized SVDs run in the same launches).
struct SmallProb {
  const float* in;    // chol: G (l x l); trsm: Y (rows x l)
  float* out;         // chol: L (l x l, lower, zeros above); trsm: Q = Y L^-T
  const float* aux;   // trsm: L
  int64_t rows;       // trsm: rows of Y
};
struct SmallBatch {
  SmallProb p[2];
  int n;
};
struct FinalProb {
  const float* M;
  const float* V;
  float* sig;   // r, descending
  float* S1;    // l x r row-major: U_s[:, :r] (x sigma if s1_sigma)
  float* S2;    // l x r row-major: V_s[:, :r] (x sigma if s2_sigma)
  int s1_sigma, s2_sigma;
  float* S1T;   // r x l row-major: S1^T (K-major operand of the tensor-core assembly)
  float* S2T;   // r x l row-major: S2^T
};
struct JacobiBatch {
  float* M[2];  // l x l column-major: in R^T, out U_s Sigma (unsorted columns)
  float* V[2];  // l x l column-major: out the accumulated rotations V_s
  int n;
  int info0;    // sweep counts go to status[1 + info0 + problem]
  float stopq;  // the cluster Jacobi stops after a sweep whose largest relative inner product is <= stopq * tol
  // r > 0: the sorted rank-r outputs of fin[] (as svd_finalize writes them)
  // are produced by the Jacobi kernel itself where it can (l <= 320)
  int r;
  FinalProb fin[2];
  // bounded waits of the cluster Jacobi's block moves (SM clock cycles), and
  // the rank of a CTA that skips its first move (-1: none; failure-path tests)
  long long wait_cycles = 1ll << 30;
  int drop_rank = -1;
};
struct FinalBatch {
  FinalProb p[2];
  int n;
};
// Cholesky G + shift_rel * max(diag G) I = L L^T.
lramm_status launch_chol(SmallBatch bt, int l, float shift_rel, int* status, cudaStream_t s);
// Q = Y L^-T.
lramm_status launch_trsm_rows(SmallBatch bt, int l, cudaStream_t s);
// One-sided Jacobi SVD of each M (thread-block cluster per problem).
// *finalized: whether the launch also wrote the sorted rank-r outputs (jb.r > 0).
lramm_status launch_jacobi(JacobiBatch jb, int l, int max_sweeps, int* status, cudaStream_t s, bool* finalized);
// The M-only pair Jacobi (l <= 544, jb.r > 0): rotates M = R^T alone and
// writes sig, S1 (as launch_jacobi does) and S2 = U_s Sigma^-1 (x sigma if
// s2_sigma) from M.  check_only: only reports in `ok` whether this shape
// launches on this device (nothing is enqueued).
lramm_status launch_jacobi_uonly(JacobiBatch jb, int l, int max_sweeps, int* status, cudaStream_t s, bool check_only,
                                 bool& ok);
// Sort by descending sigma and write the rank-r pieces.
lramm_status launch_svd_finalize(FinalBatch fb, int l, int r, cudaStream_t s);
// orth.cu -- CholeskyQR building blocks, batched over up to two problems.
struct GramProb {
  const float* Y;   // rows x l, stride l
  int64_t rows;
  float* G;         // l x l
};
struct GramBatch {
  GramProb p[2];
  int n;
};
struct CholProb {
  const float* G;   // l x l
  float* L;         // l x l, lower, zeros above
  float* Xd;        // ceil(l/32) blocks of 32 x 32: inverses of L's diagonal blocks (chol3: null = not wanted)
  // breakdown words: with brk set, a non-positive pivot stores 1 in *brk (and
  // in *brk_any) instead of latching LRAMM_ERR_NUMERIC, for a retry
  int* brk = nullptr;
  int* brk_any = nullptr;
  int* brk_count = nullptr;   // incremented once per factorisation that broke down (diagnostics)
};
struct CholBatch {
  CholProb p[2];
  int n;
};
struct TrsmProb {
  const float* Y;   // rows x l, stride l
  float* Q;         // rows x l: Y L^-T
  const float* L;
  const float* Xd;
  int64_t rows;
};
struct TrsmBatch {
  TrsmProb p[2];
  int n;
};
bool chol3_supported(int l);
// shift_big_rel > 0: on a non-positive pivot the kernel refactors with that
// larger relative shift (and sets *brk_any of the problem when given).
lramm_status launch_chol3(CholBatch cb, int l, float shift_rel, int* status, cudaStream_t s,
                          const int* cond = nullptr, float shift_big_rel = 0.f);
lramm_status launch_trsm3(TrsmBatch tb, int l, cudaStream_t s, const int* cond = nullptr);
// L^-1 of a Cholesky factor (L dense lower, l x l row-major) as TF32 high /
// low parts Lh, Ll (l x l row-major each).
struct LinvProb {
  const float* L;
  float* Lh;
  float* Ll;
};
struct LinvBatch {
  LinvProb p[2];
  int n;
};
lramm_status launch_linv(LinvBatch lb, int l, cudaStream_t s, const int* cond = nullptr);
// dst = src (n floats) when *cond != 0
lramm_status launch_copy_cond(const float* src, float* dst, int64_t n, const int* cond, cudaStream_t s);
// Two-level Cholesky for 288 < l <= 576 (l % 4 == 0) on chol3 / trsm3 /
// sgemm; scratch: chol_split_scratch_floats(l) floats per problem.
struct SplitScratch {
  float* w[2];
};
bool chol_split_supported(int l);
size_t chol_split_scratch_floats(int l);
lramm_status launch_chol_split(CholBatch cb, SplitScratch sc, int l, float shift_rel, int* status, cudaStream_t s,
                               const int* cond = nullptr);
size_t gram_part_floats(int l);
lramm_status launch_gram(GramBatch gb, int l, float* part, cudaStream_t s, const int* cond = nullptr);
lramm_status launch_chol2(SmallBatch bt, int l, float shift_rel, int* status, cudaStream_t s);
lramm_status launch_trsm_panel(SmallBatch bt, int l, cudaStream_t s);
// Range-finder backward helpers: out = copyltu(M) (lower triangle mirrored),
// I = identity (l x l), x *= a.
lramm_status launch_copyltu(const float* M, float* out, int l, cudaStream_t s);
lramm_status launch_identity(float* I, int l, cudaStream_t s);
lramm_status launch_scale(float* x, int64_t n, float a, cudaStream_t s);
lramm_status launch_axpy(float* y, const float* x, int64_t n, float a, cudaStream_t s);   // y += a x
// Largest l the small-SVD kernels accept.
int jacobi_max_l();

// qgemm_tc.cu -- code products on the tensor cores: INT8 codes as BF16
// (exact integer sums), INT4 / E4M3 codes as FP8 e4m3; fused dequantisation
// epilogue.  tgemm_tc: C = alpha A B^T + beta C with FP32 operands as TF32
// (A: M x K, B: N x K, both K-major).
bool qgemm_tc_supported(int prec, const void* L, const void* R, int64_t ldl, int64_t ldr, int64_t M, int64_t N,
                        int64_t K);
size_t qgemm_tc_part_floats(int prec, int64_t M, int64_t N, int64_t K);
lramm_status qgemm_tc(int prec, const void* L, const void* R, int64_t M, int64_t N, int64_t K, int64_t ldl,
                      int64_t ldr, int per_row, const float* sL, const float* sR, float alpha, float beta,
                      const float* C, int64_t ldc, float* D, int64_t ldd, float* part, size_t part_floats,
                      int* status, cudaStream_t s);
bool tgemm_tc_supported(const float* A, const float* B, int64_t lda, int64_t ldb, int64_t M, int64_t N, int64_t K);
// qterms_tc: D = alpha sum_t fp32(fp32(L_t R_t^T) * fp32(sL_t sR_t)) + beta C
// over up to 4 terms of BF16 operands (L_t: M x K_t, R_t: N x K_t, K-major)
// in one pass over D; sL_t = nullptr marks an unscaled term (exact BF16
// values, FP32 sums); scaled terms hold INT8 codes with K_t <= 1024.
bool qterms_tc_supported(int nterms, const void* const* L, const void* const* R, const int64_t* K, const int64_t* ldl,
                         const int64_t* ldr, const float* const* sL, int64_t M, int64_t N);
lramm_status qterms_tc(int nterms, const void* const* L, const void* const* R, const int64_t* K, const int64_t* ldl,
                       const int64_t* ldr, const float* const* sL, const float* const* sR, int per_row, int64_t M,
                       int64_t N, float alpha, float beta, const float* C, int64_t ldc, float* D, int64_t ldd,
                       int* status, cudaStream_t s);
size_t tgemm_tc_part_floats(int64_t M, int64_t N, int64_t K);
lramm_status tgemm_tc(int64_t M, int64_t N, int64_t K, float alpha, const float* A, int64_t lda, const float* B,
                      int64_t ldb, float beta, float* C, int64_t ldc, float* part, size_t part_floats, int* status,
                      cudaStream_t s);
// sketch_tc.cu -- X B / X^T B on the tensor cores (TF32, FP32 accumulate)
bool sketch_tc_supported(int xbf, int64_t ldx, int l, const void* X, const void* B);
size_t sketch_tc_part_floats(int l);
// BF16 X: B split into BF16 parts (nb = 2: hi + lo; 1: hi only), kind::f16;
// split: sketch_bf_split_bytes(K, l) bytes of scratch for the parts.
bool sketch_bf_supported(int64_t ldx, int l, const void* X, const void* B);
size_t sketch_bf_split_bytes(int64_t K, int l);
// Gram G = Y^T Y on the tensor cores in split TF32 (~2^-21 relative), one
// or two problems (Y rows x l, stride l, l % 4 == 0).
bool gram_tc_supported(int l);
size_t gram_tc_part_floats(int l);
lramm_status gram_tc(int n, const float* const* Y, const int64_t* rows, float* const* G, int l, float* part,
                     size_t part_floats, int* status, cudaStream_t s, const int* cond = nullptr);
lramm_status sketch_bf(int a_mn, const void* X, int64_t rows, int64_t cols, int64_t ldx, const float* B, int l,
                       int nb, float* out, float* part, size_t part_floats, void* split, size_t split_bytes,
                       int* status, cudaStream_t s);
lramm_status sketch_tc(int a_mn, const void* X, int64_t rows, int64_t cols, int64_t ldx, int xbf, const float* B,
                       int l, float* out, float* part, size_t part_floats, int* status, cudaStream_t s);
// Q = Y L^-T (Y rows x l, stride l; Q may be Y) in split TF32 from the parts
// Lh + Ll = L^-1 written by launch_linv; l % 4 == 0, 16 <= l <= 288.
bool basis_tc_supported(int l);
lramm_status basis_tc(const float* Y, int64_t rows, const float* Lh, const float* Ll, float* Q, int l, int* status,
                      cudaStream_t s, const int* cond = nullptr);

// quant.cu
lramm_status quantize_rows(const float* X, int64_t rows, int64_t cols, int64_t ldx, int prec,
                           int per_row, void* codes, int64_t ldcodes, float* scales,
                           unsigned int* amax_ws, cudaStream_t s);
lramm_status fp8_codes_to_bf16(const void* src, int64_t rows, int64_t cols, int64_t lds, void* dst, int64_t ldd,
                               cudaStream_t s);
// Columns of X quantised as the rows of a K-major code matrix (cols x ldcodes).
lramm_status quantize_cols(const float* X, int64_t rows, int64_t cols, int64_t ldx, int prec, int per_col,
                           void* codesT, int64_t ldcodes, float* scales, unsigned int* amax_ws, cudaStream_t s);
// The same per-column quantisation (identical codes and scales) on a 2-D
// grid of column blocks x row chunks, for tall matrices with few columns:
// amax_cols (cols words of scratch) receives the column a_max first.
lramm_status quantize_cols2d(const float* X, int64_t rows, int64_t cols, int64_t ldx, int prec, void* codesT,
                             int64_t ldcodes, float* scales, unsigned int* amax_cols, cudaStream_t s);
lramm_status quantize_rows_noalloc(const float* X, int64_t rows, int64_t cols, int64_t ldx, int prec,
                                   int per_row, void* codes, int64_t ldcodes, float* scales,
                                   cudaStream_t s);
size_t noalloc_scratch_bytes();

// mx.cu -- MXFP4 operands (unpacked codes: int8 = 2 x e2m1 value; int8 block
// exponents, one per 32 codes along K), the block-scaled QM product, and the
// residual r = x - c s of a quantised factor.
lramm_status quantize_mx(const float* X, int64_t rows, int64_t cols, int64_t ldx, int8_t* codes, int64_t ldc,
                         int8_t* exps, cudaStream_t s);
// The same decisions, each element written as its exact BF16 value q 2^e.
lramm_status quantize_mx_values(const float* X, int64_t rows, int64_t cols, int64_t ldx, __nv_bfloat16* vals,
                                int64_t ldv, cudaStream_t s);
lramm_status qgemm_mx(const int8_t* Lc, const int8_t* Le, const int8_t* Rc, const int8_t* Re, int64_t M, int64_t N,
                      int64_t K, int64_t ldl, int64_t ldr, float alpha, float beta, const float* C, int64_t ldc,
                      float* D, int64_t ldd, cudaStream_t s);
lramm_status residual_rows(const float* X, int64_t rows, int64_t cols, int64_t ldx, int prec, const void* codes,
                           int64_t ldcodes, const float* scales, int per_row, float* out, int64_t ldo,
                           cudaStream_t s);
lramm_status qgemm(const void* L, const void* Rt, int64_t M, int64_t N, int64_t K, int64_t ldl,
                   int64_t ldr, int prec, int per_row, const float* sL, const float* sR, float alpha,
                   float beta, const float* C, int64_t ldc, void* D, int64_t ldd, int out_kind,
                   cudaStream_t s);

}  // namespace lramm
