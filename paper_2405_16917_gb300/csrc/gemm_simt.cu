// FP32 SIMT GEMM, C = alpha * op(A) op(B) + beta * C, for the small and
// medium contractions of the pipeline (Gram matrices, triangular applies,
// factor assembly, unquantised factor chain) and as the FP32-accurate
// sketch product.  64 x 64 output tile per 256-thread block, 4 x 4 per
// thread, K staged through a double-buffered shared-memory tile 16 at a
// time, operands read back as float4 broadcasts.
//
// Accumulation: each 16-deep K tile is summed in a fresh FP32 register and
// added to the running sum with Kahan compensation, so the rounding error
// of an entry is ~ (4 + O(1)) u sum|a_k b_k| whatever K is (a plain FMA
// chain grows like sqrt(K) u; K reaches 32768 here).
#include "common.cuh"

namespace lramm {

template <int TA, int TB, typename TAe>
__global__ void __launch_bounds__(256)
sgemm_kernel(int64_t M, int64_t N, int64_t K, float alpha, const TAe* __restrict__ A, int64_t lda,
             const float* __restrict__ B, int64_t ldb, float beta, float* __restrict__ C,
             int64_t ldc, const int* __restrict__ cond) {
  if (cond && *cond == 0) return;   // predicated launch: the flag is unset, nothing to do
  // double-buffered K tiles: the next tile's elements are fetched into
  // registers while the current one is multiplied (one barrier per tile);
  // rows padded to 68 floats (aligned float4 reads, few store conflicts)
  __shared__ __align__(16) float As[2][16][68];
  __shared__ __align__(16) float Bs[2][16][68];
  const int tid = threadIdx.x;
  const int64_t m0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * 64;
  const int tx = tid & 15, ty = tid >> 4;
  float acc[4][4], cmp[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = cmp[i][j] = 0.f;
  float ra[4], rb[4];
  auto fetch = [&](int64_t k0) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + u * 256;
      int mm, kk;
      if (TA == 0) {  // A row-major M x K: contiguous along k
        kk = e & 15;
        mm = e >> 4;
      } else {        // A stored K x M: contiguous along m
        mm = e & 63;
        kk = e >> 6;
      }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      ra[u] = (gm < M && gk < K) ? load_as_float(TA == 0 ? A + gm * lda + gk : A + gk * lda + gm) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + u * 256;
      int nn, kk;
      if (TB == 0) {  // B row-major K x N: contiguous along n
        nn = e & 63;
        kk = e >> 6;
      } else {        // B stored N x K: contiguous along k
        kk = e & 15;
        nn = e >> 4;
      }
      const int64_t gn = n0 + nn, gk = k0 + kk;
      rb[u] = (gn < N && gk < K) ? (TB == 0 ? B[gk * ldb + gn] : B[gn * ldb + gk]) : 0.f;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + u * 256;
      if (TA == 0) As[buf][e & 15][e >> 4] = ra[u];
      else As[buf][e >> 6][e & 63] = ra[u];
      if (TB == 0) Bs[buf][e >> 6][e & 63] = rb[u];
      else Bs[buf][e & 15][e >> 4] = rb[u];
    }
  };
  if (K > 0) {
    fetch(0);
    stash(0);
  }
  __syncthreads();
  int cur = 0;
  for (int64_t k0 = 0; k0 < K; k0 += 16) {
    const bool more = k0 + 16 < K;
    if (more) fetch(k0 + 16);
    float blk[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) blk[i][j] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const float4 a4 = *reinterpret_cast<const float4*>(&As[cur][kk][ty * 4]);
      const float4 b4 = *reinterpret_cast<const float4*>(&Bs[cur][kk][tx * 4]);
      const float a[4] = {a4.x, a4.y, a4.z, a4.w};
      const float b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) blk[i][j] = fmaf(a[i], b[j], blk[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {  // Kahan: acc += blk
        const float y = blk[i][j] - cmp[i][j];
        const float t = acc[i][j] + y;
        cmp[i][j] = (t - acc[i][j]) - y;
        acc[i][j] = t;
      }
    if (more) stash(cur ^ 1);
    __syncthreads();
    cur ^= 1;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gm = m0 + ty * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      float v = alpha * acc[i][j];
      if (beta != 0.f) v = fmaf(beta, C[gm * ldc + gn], v);
      C[gm * ldc + gn] = v;
    }
  }
}

template <typename TAe>
static lramm_status sgemm_t(int ta, int tb, int64_t M, int64_t N, int64_t K, float alpha,
                            const TAe* A, int64_t lda, const float* B, int64_t ldb, float beta,
                            float* C, int64_t ldc, const int* cond, cudaStream_t s) {
  if (M <= 0 || N <= 0) return LRAMM_OK;
  if (ceil_div(M, 64) > 65535) return LRAMM_ERR_UNSUPPORTED;
  dim3 grid((unsigned)ceil_div(N, 64), (unsigned)ceil_div(M, 64));
  if (ta == 0 && tb == 0)
    sgemm_kernel<0, 0, TAe><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, cond);
  else if (ta == 0 && tb == 1)
    sgemm_kernel<0, 1, TAe><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, cond);
  else if (ta == 1 && tb == 0)
    sgemm_kernel<1, 0, TAe><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, cond);
  else
    sgemm_kernel<1, 1, TAe><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, cond);
  return last_launch();
}

lramm_status sgemm(int ta, int tb, int64_t M, int64_t N, int64_t K, float alpha, const void* A,
                   int64_t lda, int a_bf16, const float* B, int64_t ldb, float beta, float* C,
                   int64_t ldc, cudaStream_t s, const int* cond) {
  if (a_bf16)
    return sgemm_t<__nv_bfloat16>(ta, tb, M, N, K, alpha, static_cast<const __nv_bfloat16*>(A), lda,
                                  B, ldb, beta, C, ldc, cond, s);
  return sgemm_t<float>(ta, tb, M, N, K, alpha, static_cast<const float*>(A), lda, B, ldb, beta, C,
                        ldc, cond, s);
}

}  // namespace lramm
