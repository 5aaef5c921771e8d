// MXFP4 operands (e2m1 elements with one power-of-two scale per 32
// consecutive elements along K), split-precision residuals, and the
// block-scaled QM product.
//
// Quantiser (one warp per row, one lane per element of a 32-block):
//   a_max of the block (exact), e = ceil(log2(fp32(a_max / 6))) clamped to
//   [-127, 127] (-127 for an all-zero block), element = x 2^-e rounded to
//   nearest-even on the e2m1 grid {0, 0.5, 1, 1.5, 2, 3, 4, 6} (no element
//   exceeds 6 under this scale rule).  Codes are stored unpacked as int8
//   holding twice the e2m1 value (integers in [-12, 12]), exponents as int8.
// Product: acc(i,j) = sum_b 2^(eL[i,b] + eR[j,b] - 2) P_b(i,j), P_b the exact
//   integer dot product of the two 32-code blocks (4-way int8 dot products),
//   the block terms added in FP32 in block order; D = alpha acc + beta C.
// Residual of the split-precision lead factors: r = fp32(x - fp32(c s))
//   for codes c with scales s (per row or per tensor), in the code formats
//   of the quantiser in quant.cu.
#include "common.cuh"

namespace lramm {

constexpr int kMxB = 32;

__device__ __forceinline__ float warp_max_mx(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Nearest-even rounding onto the e2m1 magnitudes: the grid spacing is 0.5
// below 2, 1 in [2, 4) and 2 in [4, 8); a / spacing is exact (power of two).
__device__ __forceinline__ float round_e2m1(float y) {
  const float a = fabsf(y);
  const float inv = a < 2.f ? 2.f : (a < 4.f ? 1.f : 0.5f);
  const float r = fminf(rintf(a * inv) / inv, 6.f);
  return copysignf(r, y);
}

__device__ __forceinline__ int mx_exponent(float amax) {
  if (!(amax > 0.f)) return -127;
  const float y = __fdiv_rn(amax, 6.0f);
  int E;
  const float m = frexpf(y, &E);   // y = m 2^E, m in [0.5, 1)
  int e = m > 0.5f ? E : E - 1;    // ceil(log2 y)
  return e < -127 ? -127 : (e > 127 ? 127 : e);
}

__global__ void __launch_bounds__(256) quant_mx_kernel(const float* __restrict__ X, int64_t rows, int64_t cols,
                                                       int64_t ldx, int8_t* __restrict__ codes, int64_t ldc,
                                                       int8_t* __restrict__ exps) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  const int64_t nb = ldc / kMxB;
  for (int64_t row = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5); row < rows;
       row += warps) {
    const float* x = X + row * ldx;
    for (int64_t b = 0; b < nb; ++b) {
      const int64_t j = b * kMxB + lane;
      const float v = j < cols ? x[j] : 0.f;
      const int e = mx_exponent(warp_max_mx(fabsf(v)));
      const float q = round_e2m1(ldexpf(v, -e));
      codes[row * ldc + j] = static_cast<int8_t>(__float2int_rn(2.f * q));
      if (lane == 0) exps[row * nb + b] = static_cast<int8_t>(e);
    }
  }
}

// The same quantiser writing each element's value q 2^e as bfloat16 (K
// columns padded with zeros to ldv): q has at most two significant bits, so
// the value is exact in BF16 for every block exponent of a finite input
// (subnormal below 2^-126).  These are the operands of the tensor-core E3
// product, whose BF16 products are exact.
__global__ void __launch_bounds__(256) quant_mx_values_kernel(const float* __restrict__ X, int64_t rows, int64_t cols,
                                                              int64_t ldx, __nv_bfloat16* __restrict__ vals,
                                                              int64_t ldv) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  const int64_t nb = ldv / kMxB;
  for (int64_t row = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5); row < rows;
       row += warps) {
    const float* x = X + row * ldx;
    for (int64_t b = 0; b < nb; ++b) {
      const int64_t j = b * kMxB + lane;
      const float v = j < cols ? x[j] : 0.f;
      const int e = mx_exponent(warp_max_mx(fabsf(v)));
      const float q = round_e2m1(ldexpf(v, -e));
      vals[row * ldv + j] = __float2bfloat16_rn(ldexpf(q, e));
    }
  }
}

lramm_status quantize_mx_values(const float* X, int64_t rows, int64_t cols, int64_t ldx, __nv_bfloat16* vals,
                                int64_t ldv, cudaStream_t s) {
  if (rows <= 0) return LRAMM_OK;
  if (ldv % kMxB || ldv < cols) return LRAMM_ERR_INVALID_ARG;
  int64_t g = ceil_div(rows, 8);
  if (g > num_sms() * 16) g = num_sms() * 16;
  quant_mx_values_kernel<<<static_cast<unsigned>(g), 256, 0, s>>>(X, rows, cols, ldx, vals, ldv);
  return last_launch();
}

lramm_status quantize_mx(const float* X, int64_t rows, int64_t cols, int64_t ldx, int8_t* codes, int64_t ldc,
                         int8_t* exps, cudaStream_t s) {
  if (rows <= 0) return LRAMM_OK;
  if (ldc % kMxB || ldc < cols) return LRAMM_ERR_INVALID_ARG;
  int64_t g = ceil_div(rows, 8);
  if (g > num_sms() * 16) g = num_sms() * 16;
  quant_mx_kernel<<<static_cast<unsigned>(g), 256, 0, s>>>(X, rows, cols, ldx, codes, ldc, exps);
  return last_launch();
}

// 64 x 64 output tile per CTA, 256 threads with 4 x 4 outputs each; per
// 32-block the two code tiles (64 x 32 int8 each) and exponents are staged in
// shared memory and every thread forms its 16 exact block dot products with
// 4-way int8 dot instructions.
__global__ void __launch_bounds__(256) qgemm_mx_kernel(const int8_t* __restrict__ Lc, const int8_t* __restrict__ Le,
                                                       const int8_t* __restrict__ Rc, const int8_t* __restrict__ Re,
                                                       int64_t M, int64_t N, int64_t K, int64_t ldl, int64_t ldr,
                                                       float alpha, float beta, const float* __restrict__ C,
                                                       int64_t ldc, float* __restrict__ D, int64_t ldd) {
  __shared__ int Ls[64][9];
  __shared__ int Rs[64][9];
  __shared__ int Les[64], Res[64];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = static_cast<int64_t>(blockIdx.y) * 64, n0 = static_cast<int64_t>(blockIdx.x) * 64;
  const int64_t nb = K / kMxB;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = 0.f;
  for (int64_t b = 0; b < nb; ++b) {
    __syncthreads();
    for (int e = tid; e < 64 * 8; e += 256) {   // 8 words (32 codes) per row
      const int r = e >> 3, w = e & 7;
      const int64_t gi = m0 + r, gj = n0 + r;
      Ls[r][w] = gi < M ? reinterpret_cast<const int*>(Lc + gi * ldl + b * kMxB)[w] : 0;
      Rs[r][w] = gj < N ? reinterpret_cast<const int*>(Rc + gj * ldr + b * kMxB)[w] : 0;
    }
    if (tid < 64) {
      Les[tid] = m0 + tid < M ? Le[(m0 + tid) * nb + b] : 0;
    } else if (tid < 128) {
      const int t = tid - 64;
      Res[t] = n0 + t < N ? Re[(n0 + t) * nb + b] : 0;
    }
    __syncthreads();
    int p[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) p[a][c] = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      int lw[4], rw[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) lw[a] = Ls[ty * 4 + a][w];
#pragma unroll
      for (int c = 0; c < 4; ++c) rw[c] = Rs[tx * 4 + c][w];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) p[a][c] = __dp4a(lw[a], rw[c], p[a][c]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c)
        acc[a][c] += ldexpf(static_cast<float>(p[a][c]), Les[ty * 4 + a] + Res[tx * 4 + c] - 2);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t i = m0 + ty * 4 + a;
    if (i >= M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t j = n0 + tx * 4 + c;
      if (j >= N) continue;
      float o = __fmul_rn(alpha, acc[a][c]);
      if (beta != 0.f) o = fmaf(beta, C[i * ldc + j], o);
      D[i * ldd + j] = o;
    }
  }
}

lramm_status qgemm_mx(const int8_t* Lc, const int8_t* Le, const int8_t* Rc, const int8_t* Re, int64_t M, int64_t N,
                      int64_t K, int64_t ldl, int64_t ldr, float alpha, float beta, const float* C, int64_t ldc,
                      float* D, int64_t ldd, cudaStream_t s) {
  if (M <= 0 || N <= 0) return LRAMM_OK;
  if (K % kMxB || ldl % 16 || ldr % 16 || ldl < K || ldr < K) return LRAMM_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(Lc) | reinterpret_cast<uintptr_t>(Rc)) & 15) return LRAMM_ERR_INVALID_ARG;
  if (ceil_div(M, 64) > 65535) return LRAMM_ERR_UNSUPPORTED;
  qgemm_mx_kernel<<<dim3(static_cast<unsigned>(ceil_div(N, 64)), static_cast<unsigned>(ceil_div(M, 64))), 256, 0, s>>>(
      Lc, Le, Rc, Re, M, N, K, ldl, ldr, alpha, beta, C, ldc, D, ldd);
  return last_launch();
}

// r = fp32(x - fp32(c s)) for codes c (container by precision) with scales s.
template <int CT>
__global__ void resid_kernel(const float* __restrict__ X, int64_t rows, int64_t cols, int64_t ldx,
                             const void* __restrict__ codes, int64_t ldcodes, const float* __restrict__ scales,
                             int per_row, float* __restrict__ out, int64_t ldo) {
  const int64_t n = rows * cols;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / cols, j = e - i * cols;
    const float c = CT == CODE_BF16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(codes)[i * ldcodes + j])
                                    : e4m3_to_float(static_cast<const uint8_t*>(codes)[i * ldcodes + j]);
    const float s = per_row ? scales[i] : scales[0];
    out[i * ldo + j] = __fsub_rn(X[i * ldx + j], __fmul_rn(c, s));
  }
}

lramm_status residual_rows(const float* X, int64_t rows, int64_t cols, int64_t ldx, int prec, const void* codes,
                           int64_t ldcodes, const float* scales, int per_row, float* out, int64_t ldo,
                           cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return LRAMM_OK;
  int64_t g = ceil_div(rows * cols, 256);
  if (g > num_sms() * 8) g = num_sms() * 8;
  if (code_type_of(prec) == CODE_BF16)
    resid_kernel<CODE_BF16><<<static_cast<unsigned>(g), 256, 0, s>>>(X, rows, cols, ldx, codes, ldcodes, scales,
                                                                      per_row, out, ldo);
  else
    resid_kernel<CODE_E4M3><<<static_cast<unsigned>(g), 256, 0, s>>>(X, rows, cols, ldx, codes, ldcodes, scales,
                                                                      per_row, out, ldo);
  return last_launch();
}

}  // namespace lramm
