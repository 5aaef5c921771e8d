// Symmetric linear quantiser (Eqs. (Quantization), (get_lambda), Sec. 3.1)
// and the quantised GEMM QM of Algorithm 2 with a fused FP32 dequantisation
// (Eq. (Dequantization)) and the alpha/beta epilogue of Algorithm 3.
//
// The decisions are taken in FP32: a_max exact, lambda = D / a_max (IEEE
// division), code = rint(x * lambda) (one FP32 multiply, round half to even)
// clamped to +-D; e4m3 codes are the round-to-nearest-even, saturating FP8
// conversion of x * lambda.  Dequantisation of a product entry:
//   fp32(acc) * fp32(s_left[i] * s_right[j]),  s = a_max / D.
#include <mutex>

#include "common.cuh"

namespace lramm {

__device__ __forceinline__ float warp_max_q(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Whole-tensor a_max into *amax (as the bits of a non-negative float, so an
// unsigned atomicMax orders them correctly).  *amax must start at 0.
__global__ void tensor_amax_kernel(const float* __restrict__ X, int64_t rows, int64_t cols, int64_t ldx,
                                   unsigned int* amax) {
  float m = 0.f;
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e - i * cols;
    m = fmaxf(m, fabsf(X[i * ldx + j]));
  }
  m = warp_max_q(m);
  if ((threadIdx.x & 31) == 0) atomicMax(amax, __float_as_uint(m));
}

template <int PREC>
__device__ __forceinline__ void store_code(void* codes, int64_t idx, float y, float D) {
  if (PREC == LRAMM_P_E4M3) {
    static_cast<uint8_t*>(codes)[idx] = __nv_cvt_float_to_fp8(y, __NV_SATFINITE, __NV_E4M3);
  } else {
    const float v = fminf(fmaxf(rintf(y), -D), D);
    if (PREC == LRAMM_P_INT8)
      static_cast<__nv_bfloat16*>(codes)[idx] = __float2bfloat16_rn(v);
    else
      static_cast<uint8_t*>(codes)[idx] = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
  }
}

// One warp per row.  Per-row mode finds the row's a_max; per-tensor mode
// reads the whole-tensor a_max from *tensor_amax.
template <int PREC>
__global__ void quant_rows_kernel(const float* __restrict__ X, int64_t rows, int64_t cols, int64_t ldx,
                                  void* __restrict__ codes, int64_t ldcodes, float* __restrict__ scales,
                                  const unsigned int* __restrict__ tensor_amax) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const float D = PREC == LRAMM_P_INT8 ? 127.0f : (PREC == LRAMM_P_INT4 ? 7.0f : 448.0f);
  for (int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); row < rows;
       row += warps) {
    const float* x = X + row * ldx;
    float amax;
    if (tensor_amax) {
      amax = __uint_as_float(*tensor_amax);
    } else {
      amax = 0.f;
      for (int64_t j = lane; j < cols; j += 32) amax = fmaxf(amax, fabsf(x[j]));
      amax = warp_max_q(amax);
    }
    const float lam = amax > 0.f ? __fdiv_rn(D, amax) : 0.f;
    if (lane == 0 && (tensor_amax == nullptr || row == 0))
      scales[tensor_amax ? 0 : row] = __fdiv_rn(amax, D);
    for (int64_t j = lane; j < ldcodes; j += 32) {
      const float y = j < cols ? __fmul_rn(x[j], lam) : 0.f;
      store_code<PREC>(codes, row * ldcodes + j, y, D);
    }
  }
}

lramm_status quantize_rows(const float* X, int64_t rows, int64_t cols, int64_t ldx, int prec,
                           int per_row, void* codes, int64_t ldcodes, float* scales,
                           unsigned int* amax_ws, cudaStream_t s) {
  if (rows <= 0) return LRAMM_OK;
  const unsigned int* tam = nullptr;
  if (!per_row) {
    if (!amax_ws) return LRAMM_ERR_INVALID_ARG;
    LRAMM_CUDA_TRY(cudaMemsetAsync(amax_ws, 0, sizeof(unsigned int), s));
    int64_t g = ceil_div(rows * cols, 256);
    if (g > num_sms() * 8) g = num_sms() * 8;
    if (g < 1) g = 1;
    tensor_amax_kernel<<<(unsigned)g, 256, 0, s>>>(X, rows, cols, ldx, amax_ws);
    LRAMM_TRY(last_launch());
    tam = amax_ws;
  }
  const int threads = 256, wpb = threads / 32;
  int64_t g = ceil_div(rows, wpb);
  if (g > num_sms() * 16) g = num_sms() * 16;
  switch (prec) {
    case LRAMM_P_INT8:
      quant_rows_kernel<LRAMM_P_INT8><<<(unsigned)g, threads, 0, s>>>(X, rows, cols, ldx, codes, ldcodes, scales, tam);
      break;
    case LRAMM_P_INT4:
      quant_rows_kernel<LRAMM_P_INT4><<<(unsigned)g, threads, 0, s>>>(X, rows, cols, ldx, codes, ldcodes, scales, tam);
      break;
    case LRAMM_P_E4M3:
      quant_rows_kernel<LRAMM_P_E4M3><<<(unsigned)g, threads, 0, s>>>(X, rows, cols, ldx, codes, ldcodes, scales, tam);
      break;
    default:
      return LRAMM_ERR_INVALID_ARG;
  }
  return last_launch();
}

// e4m3 code bytes (INT4 codes, integers |c| <= 7) rewritten as bfloat16
// values, so that they meet INT8 codes in one BF16 product; every e4m3 value
// is exact in bfloat16.  Columns cols .. ldd-1 of dst are not written.
__global__ void fp8_to_bf16_kernel(const uint8_t* __restrict__ src, int64_t rows, int64_t cols, int64_t lds,
                                   __nv_bfloat16* __restrict__ dst, int64_t ldd) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e - i * cols;
    __nv_fp8_e4m3 v;
    v.__x = src[i * lds + j];
    dst[i * ldd + j] = __float2bfloat16_rn(static_cast<float>(v));
  }
}

lramm_status fp8_codes_to_bf16(const void* src, int64_t rows, int64_t cols, int64_t lds, void* dst, int64_t ldd,
                               cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return LRAMM_OK;
  int64_t g = ceil_div(rows * cols, 256);
  if (g > num_sms() * 8) g = num_sms() * 8;
  fp8_to_bf16_kernel<<<(unsigned)g, 256, 0, s>>>(static_cast<const uint8_t*>(src), rows, cols, lds,
                                                 static_cast<__nv_bfloat16*>(dst), ldd);
  return last_launch();
}

// Column quantiser: the columns of X (rows x cols, row-major) become the
// rows of a K-major code matrix codesT (cols x ldcodes, ldcodes >= rows,
// zero beyond rows) with one scale per column (or the tensor a_max) --
// the right operand of a direct QM(A B).  One CTA per 32 columns: pass 1
// finds each column's a_max (8 warps over the rows, coalesced rows of 32),
// pass 2 quantises 32 x 32 tiles and writes them transposed through shared
// memory.  Same FP32 decisions as quant_rows_kernel.
template <int PREC>
__global__ void __launch_bounds__(256) quant_cols_kernel(const float* __restrict__ X, int64_t rows, int64_t cols,
                                                         int64_t ldx, void* __restrict__ codesT, int64_t ldcodes,
                                                         float* __restrict__ scales,
                                                         const unsigned int* __restrict__ tensor_amax) {
  __shared__ float s_am[8][32];
  __shared__ float s_lam[32];
  __shared__ float tile[32][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * 32;
  const int64_t col = c0 + lane;
  const float D = PREC == LRAMM_P_INT8 ? 127.0f : (PREC == LRAMM_P_INT4 ? 7.0f : 448.0f);
  if (tensor_amax) {
    if (warp == 0) s_am[0][lane] = __uint_as_float(*tensor_amax);
  } else {
    float am = 0.f;
    if (col < cols)
      for (int64_t r = warp; r < rows; r += 8) am = fmaxf(am, fabsf(X[r * ldx + col]));
    s_am[warp][lane] = am;
  }
  __syncthreads();
  if (warp == 0) {
    float am = s_am[0][lane];
    if (!tensor_amax)
      for (int w = 1; w < 8; ++w) am = fmaxf(am, s_am[w][lane]);
    s_lam[lane] = am > 0.f ? __fdiv_rn(D, am) : 0.f;
    if (col < cols && (tensor_amax == nullptr || col == 0)) scales[tensor_amax ? 0 : col] = __fdiv_rn(am, D);
  }
  __syncthreads();
  for (int64_t r0 = 0; r0 < ldcodes; r0 += 32) {
    // load 32 rows x 32 columns (row r0 + warp + 8 i, column lane)
    for (int i = warp; i < 32; i += 8) {
      const int64_t r = r0 + i;
      tile[i][lane] = (r < rows && col < cols) ? X[r * ldx + col] : 0.f;
    }
    __syncthreads();
    // write column c0 + j (a row of codesT): lane = row offset within the tile
    for (int j = warp; j < 32; j += 8) {
      const int64_t c = c0 + j;
      const int64_t r = r0 + lane;
      if (c < cols && r < ldcodes) {
        const float y = r < rows ? __fmul_rn(tile[lane][j], s_lam[j]) : 0.f;
        store_code<PREC>(codesT, c * ldcodes + r, y, D);
      }
    }
    __syncthreads();
  }
}

lramm_status quantize_cols(const float* X, int64_t rows, int64_t cols, int64_t ldx, int prec, int per_col,
                           void* codesT, int64_t ldcodes, float* scales, unsigned int* amax_ws, cudaStream_t s) {
  if (cols <= 0) return LRAMM_OK;
  if (ldcodes < rows) return LRAMM_ERR_INVALID_ARG;
  const unsigned int* tam = nullptr;
  if (!per_col) {
    if (!amax_ws) return LRAMM_ERR_INVALID_ARG;
    LRAMM_CUDA_TRY(cudaMemsetAsync(amax_ws, 0, sizeof(unsigned int), s));
    int64_t g = ceil_div(rows * cols, 256);
    if (g > num_sms() * 8) g = num_sms() * 8;
    if (g < 1) g = 1;
    tensor_amax_kernel<<<(unsigned)g, 256, 0, s>>>(X, rows, cols, ldx, amax_ws);
    LRAMM_TRY(last_launch());
    tam = amax_ws;
  }
  const unsigned g = static_cast<unsigned>(ceil_div(cols, 32));
  switch (prec) {
    case LRAMM_P_INT8:
      quant_cols_kernel<LRAMM_P_INT8><<<g, 256, 0, s>>>(X, rows, cols, ldx, codesT, ldcodes, scales, tam);
      break;
    case LRAMM_P_INT4:
      quant_cols_kernel<LRAMM_P_INT4><<<g, 256, 0, s>>>(X, rows, cols, ldx, codesT, ldcodes, scales, tam);
      break;
    case LRAMM_P_E4M3:
      quant_cols_kernel<LRAMM_P_E4M3><<<g, 256, 0, s>>>(X, rows, cols, ldx, codesT, ldcodes, scales, tam);
      break;
    default:
      return LRAMM_ERR_INVALID_ARG;
  }
  return last_launch();
}

// Column a_max over a chunk of rows, merged across CTAs by atomicMax on the
// float bits (non-negative floats order like their bit patterns).
__global__ void __launch_bounds__(256) col_amax_kernel(const float* __restrict__ X, int64_t rows, int64_t cols,
                                                       int64_t ldx, int64_t rchunk, unsigned int* __restrict__ amax) {
  __shared__ float s_am[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t col = static_cast<int64_t>(blockIdx.x) * 32 + lane;
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * rchunk;
  const int64_t r1 = r0 + rchunk < rows ? r0 + rchunk : rows;
  float am = 0.f;
  if (col < cols)
    for (int64_t r = r0 + warp; r < r1; r += 8) am = fmaxf(am, fabsf(X[r * ldx + col]));
  s_am[warp][lane] = am;
  __syncthreads();
  if (warp == 0) {
    for (int w = 1; w < 8; ++w) am = fmaxf(am, s_am[w][lane]);
    if (col < cols) atomicMax(amax + col, __float_as_uint(am));
  }
}

// Codes of rows r0 .. r0 + rchunk - 1 (up to ldcodes, zero beyond rows) of
// 32 columns, written transposed; the column's lambda and scale as in
// quant_cols_kernel.
template <int PREC>
__global__ void __launch_bounds__(256) quant_cols2d_kernel(const float* __restrict__ X, int64_t rows, int64_t cols,
                                                           int64_t ldx, int64_t rchunk,
                                                           const unsigned int* __restrict__ amax,
                                                           void* __restrict__ codesT, int64_t ldcodes,
                                                           float* __restrict__ scales) {
  __shared__ float s_lam[32];
  __shared__ float tile[32][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * 32;
  const int64_t col = c0 + lane;
  const float D = PREC == LRAMM_P_INT8 ? 127.0f : (PREC == LRAMM_P_INT4 ? 7.0f : 448.0f);
  if (warp == 0) {
    const float am = col < cols ? __uint_as_float(amax[col]) : 0.f;
    s_lam[lane] = am > 0.f ? __fdiv_rn(D, am) : 0.f;
    if (blockIdx.y == 0 && col < cols) scales[col] = __fdiv_rn(am, D);
  }
  __syncthreads();
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * rchunk;
  const int64_t r1 = r0 + rchunk < ldcodes ? r0 + rchunk : ldcodes;
  for (int64_t rb = r0; rb < r1; rb += 32) {
    for (int i = warp; i < 32; i += 8) {
      const int64_t r = rb + i;
      tile[i][lane] = (r < rows && col < cols) ? X[r * ldx + col] : 0.f;
    }
    __syncthreads();
    for (int j = warp; j < 32; j += 8) {
      const int64_t c = c0 + j;
      const int64_t r = rb + lane;
      if (c < cols && r < r1) {
        const float y = r < rows ? __fmul_rn(tile[lane][j], s_lam[j]) : 0.f;
        store_code<PREC>(codesT, c * ldcodes + r, y, D);
      }
    }
    __syncthreads();
  }
}

lramm_status quantize_cols2d(const float* X, int64_t rows, int64_t cols, int64_t ldx, int prec, void* codesT,
                             int64_t ldcodes, float* scales, unsigned int* amax_cols, cudaStream_t s) {
  if (cols <= 0) return LRAMM_OK;
  if (ldcodes < rows || !amax_cols) return LRAMM_ERR_INVALID_ARG;
  const int64_t cblocks = ceil_div(cols, 32);
  // row chunks (multiples of 32) so that the grid has about two CTAs per SM
  int64_t nchunks = ceil_div(2 * num_sms(), cblocks);
  int64_t rchunk = round_up(ceil_div(ldcodes, nchunks), 32);
  if (rchunk < 32) rchunk = 32;
  nchunks = ceil_div(ldcodes, rchunk);
  LRAMM_CUDA_TRY(cudaMemsetAsync(amax_cols, 0, sizeof(unsigned int) * cols, s));
  col_amax_kernel<<<dim3((unsigned)cblocks, (unsigned)ceil_div(rows, rchunk)), 256, 0, s>>>(X, rows, cols, ldx, rchunk,
                                                                                            amax_cols);
  LRAMM_TRY(last_launch());
  const dim3 g((unsigned)cblocks, (unsigned)nchunks);
  switch (prec) {
    case LRAMM_P_INT8:
      quant_cols2d_kernel<LRAMM_P_INT8><<<g, 256, 0, s>>>(X, rows, cols, ldx, rchunk, amax_cols, codesT, ldcodes, scales);
      break;
    case LRAMM_P_INT4:
      quant_cols2d_kernel<LRAMM_P_INT4><<<g, 256, 0, s>>>(X, rows, cols, ldx, rchunk, amax_cols, codesT, ldcodes, scales);
      break;
    case LRAMM_P_E4M3:
      quant_cols2d_kernel<LRAMM_P_E4M3><<<g, 256, 0, s>>>(X, rows, cols, ldx, rchunk, amax_cols, codesT, ldcodes, scales);
      break;
    default:
      return LRAMM_ERR_INVALID_ARG;
  }
  return last_launch();
}

// ---------------------------------------------------------------------------
// QM product, SIMT: acc(i,j) = sum_t L(i,t) Rt(j,t) with both operands
// K-major code matrices.  Integer codes accumulate exactly: FP32 partial
// sums of at most 1024 products (|sum| <= 1024 * 127^2 < 2^24) are moved
// into an int32 accumulator.
// ---------------------------------------------------------------------------
template <int CT>
__device__ __forceinline__ float load_code(const void* p, int64_t idx) {
  if (CT == CODE_BF16) return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[idx]);
  return e4m3_to_float(static_cast<const uint8_t*>(p)[idx]);
}

template <int CT, bool EXACT>
__global__ void __launch_bounds__(256)
qgemm_simt_kernel(const void* __restrict__ Lc, const void* __restrict__ Rc, int64_t M, int64_t N, int64_t K,
                  int64_t ldl, int64_t ldr, int per_row, const float* __restrict__ sL,
                  const float* __restrict__ sR, float alpha, float beta, const float* __restrict__ C,
                  int64_t ldc, void* __restrict__ D, int64_t ldd, int out_kind) {
  __shared__ float As[32][64 + 4];
  __shared__ float Bs[32][64 + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * 64;
  float acc[4][4];
  int iacc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      acc[i][j] = 0.f;
      iacc[i][j] = 0;
    }
  int chunk = 0;
  for (int64_t k0 = 0; k0 < K; k0 += 32) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + u * 256;
      const int kk = e & 31, rr = e >> 5;
      const int64_t gk = k0 + kk;
      const int64_t gm = m0 + rr, gn = n0 + rr;
      As[kk][rr] = (gm < M && gk < K) ? load_code<CT>(Lc, gm * ldl + gk) : 0.f;
      Bs[kk][rr] = (gn < N && gk < K) ? load_code<CT>(Rc, gn * ldr + gk) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 32; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
    if (EXACT && ++chunk == 32) {  // 32 * 32 = 1024 products per FP32 partial
      chunk = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          iacc[i][j] += __float2int_rn(acc[i][j]);
          acc[i][j] = 0.f;
        }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gm = m0 + ty * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      if (EXACT) {
        const int tot = iacc[i][j] + __float2int_rn(acc[i][j]);
        if (out_kind == 1) {
          static_cast<int*>(D)[gm * ldd + gn] = tot;
          continue;
        }
        acc[i][j] = (float)tot;  // cvt.rn.f32.s32
      } else if (out_kind == 1) {
        static_cast<float*>(D)[gm * ldd + gn] = acc[i][j];
        continue;
      }
      const float sp = __fmul_rn(per_row ? sL[gm] : sL[0], per_row ? sR[gn] : sR[0]);
      const float deq = __fmul_rn(acc[i][j], sp);
      float v = __fmul_rn(alpha, deq);
      if (beta != 0.f) v = fmaf(beta, C[gm * ldc + gn], v);
      static_cast<float*>(D)[gm * ldd + gn] = v;
    }
  }
}

lramm_status qgemm(const void* L, const void* Rt, int64_t M, int64_t N, int64_t K, int64_t ldl,
                   int64_t ldr, int prec, int per_row, const float* sL, const float* sR, float alpha,
                   float beta, const float* C, int64_t ldc, void* D, int64_t ldd, int out_kind,
                   cudaStream_t s) {
  if (M <= 0 || N <= 0) return LRAMM_OK;
  if (ceil_div(M, 64) > 65535) return LRAMM_ERR_UNSUPPORTED;
  dim3 grid((unsigned)ceil_div(N, 64), (unsigned)ceil_div(M, 64));
  if (prec == LRAMM_P_INT8)
    qgemm_simt_kernel<CODE_BF16, true><<<grid, 256, 0, s>>>(L, Rt, M, N, K, ldl, ldr, per_row, sL, sR, alpha,
                                                           beta, C, ldc, D, ldd, out_kind);
  else if (prec == LRAMM_P_INT4)
    qgemm_simt_kernel<CODE_E4M3, true><<<grid, 256, 0, s>>>(L, Rt, M, N, K, ldl, ldr, per_row, sL, sR, alpha,
                                                           beta, C, ldc, D, ldd, out_kind);
  else if (prec == LRAMM_P_E4M3)
    qgemm_simt_kernel<CODE_E4M3, false><<<grid, 256, 0, s>>>(L, Rt, M, N, K, ldl, ldr, per_row, sL, sR, alpha,
                                                            beta, C, ldc, D, ldd, out_kind);
  else
    return LRAMM_ERR_INVALID_ARG;
  return last_launch();
}

// ---------------------------------------------------------------------------
// Allocation-free form of the quantiser, for callers that cannot allocate
// device memory themselves.  Per-tensor mode needs one 32-bit a_max
// accumulator; here it lives in this file's own device array instead of a
// caller-supplied workspace.  The array is part of the library image, so
// every GPU the library is loaded on holds its 256 bytes until the process
// exits.  Its device address is looked up once per device (first call on
// that device, with the device current) and handed to the kernels.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned int g_noalloc_scratch[64];
static void* g_noalloc_ptr[256];
static std::mutex g_noalloc_mu;

static lramm_status noalloc_scratch(unsigned int** out) {
  int dev = 0;
  LRAMM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return LRAMM_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    LRAMM_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = p;
  }
  *out = static_cast<unsigned int*>(g_noalloc_ptr[dev]);
  return LRAMM_OK;
}

// Scratch bytes the allocation-free quantiser may use (the size of the array).
size_t noalloc_scratch_bytes() { return sizeof(g_noalloc_scratch); }

lramm_status quantize_rows_noalloc(const float* X, int64_t rows, int64_t cols, int64_t ldx, int prec,
                                   int per_row, void* codes, int64_t ldcodes, float* scales,
                                   cudaStream_t s) {
  unsigned int* am = nullptr;
  if (!per_row && rows > 0) {
    // one accumulator per call; cleared by quantize_rows before its kernels run
    const size_t need = sizeof(unsigned int);
    if (need > sizeof(g_noalloc_scratch)) return LRAMM_ERR_UNSUPPORTED;
    LRAMM_TRY(noalloc_scratch(&am));
  }
  return quantize_rows(X, rows, cols, ldx, prec, per_row, codes, ldcodes, scales, am, s);
}

}  // namespace lramm
