// FP32 SIMT GEMM, C = alpha * op(A) op(B) + beta * C, for the small and
// medium contractions of the pipeline (Gram matrices, triangular applies,
// factor assembly, unquantised factor chain) and as the FP32-accurate
// sketch product.  64 x 64 (or, for small products, 32 x 32) output tile
// per 256-thread block, 4 x 4 (2 x 2) per thread, K staged through a
// double-buffered shared-memory tile 16 at a time, operands read back as
// vector broadcasts.
//
// Accumulation: each 16-deep K tile is summed in a fresh FP32 register and
// added to the running sum with Kahan compensation, so the rounding error
// of an entry is ~ (4 + O(1)) u sum|a_k b_k| whatever K is (a plain FMA
// chain grows like sqrt(K) u; K reaches 32768 here).
#include "common.cuh"

namespace lramm {

template <int TA, int TB, typename TAe, int T = 64>
__global__ void __launch_bounds__(256)
sgemm_kernel(int64_t M, int64_t N, int64_t K, float alpha, const TAe* __restrict__ A, int64_t lda,
             const float* __restrict__ B, int64_t ldb, float beta, float* __restrict__ C,
             int64_t ldc, const int* __restrict__ cond) {
  if (cond && *cond == 0) return;   // predicated launch: the flag is unset, nothing to do
  // T x T output tile (64, or 32 for small products: more CTAs, the same
  // arithmetic per entry), R x R per thread.  Double-buffered K tiles: the
  // next tile's elements are fetched into registers while the current one is
  // multiplied (one barrier per tile); rows padded to T + 4 floats (aligned
  // vector reads, few store conflicts)
  constexpr int R = T / 16, NF = T / 16;   // entries per thread and side; fetched elements per thread and operand
  __shared__ __align__(16) float As[2][16][T + 4];
  __shared__ __align__(16) float Bs[2][16][T + 4];
  const int tid = threadIdx.x;
  const int64_t m0 = (int64_t)blockIdx.y * T, n0 = (int64_t)blockIdx.x * T;
  const int tx = tid & 15, ty = tid >> 4;
  float acc[R][R], cmp[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = cmp[i][j] = 0.f;
  float ra[NF], rb[NF];
  auto fetch = [&](int64_t k0) {
#pragma unroll
    for (int u = 0; u < NF; ++u) {
      const int e = tid + u * 256;
      int mm, kk;
      if (TA == 0) {  // A row-major M x K: contiguous along k
        kk = e & 15;
        mm = e >> 4;
      } else {        // A stored K x M: contiguous along m
        mm = e % T;
        kk = e / T;
      }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      ra[u] = (gm < M && gk < K) ? load_as_float(TA == 0 ? A + gm * lda + gk : A + gk * lda + gm) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < NF; ++u) {
      const int e = tid + u * 256;
      int nn, kk;
      if (TB == 0) {  // B row-major K x N: contiguous along n
        nn = e % T;
        kk = e / T;
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
    for (int u = 0; u < NF; ++u) {
      const int e = tid + u * 256;
      if (TA == 0) As[buf][e & 15][e >> 4] = ra[u];
      else As[buf][e / T][e % T] = ra[u];
      if (TB == 0) Bs[buf][e / T][e % T] = rb[u];
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
    float blk[R][R];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j) blk[i][j] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[R], b[R];
      if (R == 4) {
        const float4 a4 = *reinterpret_cast<const float4*>(&As[cur][kk][ty * R]);
        const float4 b4 = *reinterpret_cast<const float4*>(&Bs[cur][kk][tx * R]);
        a[0] = a4.x, a[1] = a4.y, a[R > 2 ? 2 : 0] = a4.z, a[R > 3 ? 3 : 0] = a4.w;
        b[0] = b4.x, b[1] = b4.y, b[R > 2 ? 2 : 0] = b4.z, b[R > 3 ? 3 : 0] = b4.w;
      } else {
        const float2 a2 = *reinterpret_cast<const float2*>(&As[cur][kk][ty * R]);
        const float2 b2 = *reinterpret_cast<const float2*>(&Bs[cur][kk][tx * R]);
        a[0] = a2.x, a[1] = a2.y;
        b[0] = b2.x, b[1] = b2.y;
      }
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) blk[i][j] = fmaf(a[i], b[j], blk[i][j]);
    }
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j) {  // Kahan: acc += blk
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
  for (int i = 0; i < R; ++i) {
    const int64_t gm = m0 + ty * R + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int64_t gn = n0 + tx * R + j;
      if (gn >= N) continue;
      float v = alpha * acc[i][j];
      if (beta != 0.f) v = fmaf(beta, C[gm * ldc + gn], v);
      C[gm * ldc + gn] = v;
    }
  }
}

template <typename TAe, int T>
static lramm_status sgemm_launch(int ta, int tb, int64_t M, int64_t N, int64_t K, float alpha, const TAe* A,
                                 int64_t lda, const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                                 const int* cond, cudaStream_t s) {
  if (ceil_div(M, T) > 65535) return LRAMM_ERR_UNSUPPORTED;
  dim3 grid((unsigned)ceil_div(N, T), (unsigned)ceil_div(M, T));
  if (ta == 0 && tb == 0)
    sgemm_kernel<0, 0, TAe, T><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, cond);
  else if (ta == 0 && tb == 1)
    sgemm_kernel<0, 1, TAe, T><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, cond);
  else if (ta == 1 && tb == 0)
    sgemm_kernel<1, 0, TAe, T><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, cond);
  else
    sgemm_kernel<1, 1, TAe, T><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, cond);
  return last_launch();
}

// 32 x 32 tiles when 64 x 64 tiles would cover under half the SMs (the
// l x l products of the small SVD's neighbourhood): four times the CTAs,
// each entry computed by the same operations.
template <typename TAe>
static lramm_status sgemm_t(int ta, int tb, int64_t M, int64_t N, int64_t K, float alpha,
                            const TAe* A, int64_t lda, const float* B, int64_t ldb, float beta,
                            float* C, int64_t ldc, const int* cond, cudaStream_t s) {
  if (M <= 0 || N <= 0) return LRAMM_OK;
  if (ceil_div(M, 64) * ceil_div(N, 64) < num_sms() / 2)
    return sgemm_launch<TAe, 32>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, cond, s);
  return sgemm_launch<TAe, 64>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, cond, s);
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
