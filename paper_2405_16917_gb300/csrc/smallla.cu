// Small dense linear algebra of the randomized SVD (sizes l x l, l = r + p):
//   * Cholesky of the Gram matrix for CholeskyQR (orthonormalisation of the
//     sketch, Sec. 2.2: "a matrix Q with r orthonormal columns"),
//   * the triangular solve Q = Y L^-T that applies it to the tall sketch,
//   * one-sided Jacobi SVD of the l x l triangular factor (the SVD of
//     B = Q^* A in Algorithm 1, taken on the R factor of B^T = P R),
//   * sorting / truncation of the SVD to rank r.
// All FP32.  Every loop has a fixed trip count; nothing waits on a flag.
#include <float.h>

#include "common.cuh"

namespace lramm {

__device__ __forceinline__ int pidx(int i, int j) { return i * (i + 1) / 2 + j; }  // packed lower

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---------------------------------------------------------------------------
// Cholesky G + shift I = L L^T, G l x l row-major; packed lower triangle in
// shared memory, right-looking.  A non-positive pivot latches
// LRAMM_ERR_NUMERIC and is replaced by a tiny positive value so the
// factorisation (and everything after it) still terminates.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) chol_kernel(const float* __restrict__ G, int l,
                                                    float shift_rel, float* __restrict__ L,
                                                    int* status) {
  extern __shared__ float P[];
  __shared__ float s_red[32];
  __shared__ float s_piv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;

  float md = 0.f;
  for (int i = tid; i < l; i += blockDim.x) md = fmaxf(md, G[(int64_t)i * l + i]);
  md = warp_max(md);
  if (lane == 0) s_red[warp] = md;
  __syncthreads();
  if (warp == 0) {
    float v = lane < nw ? s_red[lane] : 0.f;
    v = warp_max(v);
    if (lane == 0) s_red[0] = v;
  }
  __syncthreads();
  const float shift = shift_rel * s_red[0];
  for (int i = warp; i < l; i += nw)
    for (int j = lane; j <= i; j += 32)
      P[pidx(i, j)] = G[(int64_t)i * l + j] + (i == j ? shift : 0.f);
  __syncthreads();

  for (int j = 0; j < l; ++j) {
    if (tid == 0) {
      float d = P[pidx(j, j)];
      if (!(d > 0.f)) {
        set_status(status, LRAMM_ERR_NUMERIC);
        d = FLT_MIN * 1024.f;
      }
      d = sqrtf(d);
      P[pidx(j, j)] = d;
      s_piv = 1.0f / d;
    }
    __syncthreads();
    const float inv = s_piv;
    for (int i = j + 1 + tid; i < l; i += blockDim.x) P[pidx(i, j)] *= inv;
    __syncthreads();
    for (int i = j + 1 + warp; i < l; i += nw) {
      const float lij = P[pidx(i, j)];
      for (int c = j + 1 + lane; c <= i; c += 32) P[pidx(i, c)] -= lij * P[pidx(c, j)];
    }
    __syncthreads();
  }
  for (int64_t e = tid; e < (int64_t)l * l; e += blockDim.x) {
    const int i = (int)(e / l), j = (int)(e - (int64_t)i * l);
    L[e] = j <= i ? P[pidx(i, j)] : 0.f;
  }
}

// ---------------------------------------------------------------------------
// Q = Y L^-T row by row: q_i = (y_i - sum_{j<i} q_j L_ij) / L_ii.
// One warp per row; L (packed) and a per-warp row buffer in shared memory.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) trsm_rows_kernel(const float* __restrict__ Y, int64_t rows,
                                                         int l, const float* __restrict__ L,
                                                         float* __restrict__ Q) {
  extern __shared__ float sm[];
  const int np = l * (l + 1) / 2;
  float* Lp = sm;
  float* dinv = sm + np;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  float* qb = dinv + l + warp * l;
  for (int i = warp; i < l; i += nw)
    for (int j = lane; j <= i; j += 32) Lp[pidx(i, j)] = L[(int64_t)i * l + j];
  __syncthreads();
  for (int i = tid; i < l; i += blockDim.x) dinv[i] = 1.0f / Lp[pidx(i, i)];
  __syncthreads();
  for (int64_t row = (int64_t)blockIdx.x * nw + warp; row < rows; row += (int64_t)gridDim.x * nw) {
    for (int i = lane; i < l; i += 32) qb[i] = Y[row * l + i];
    __syncwarp();
    for (int i = 0; i < l; ++i) {
      float part = 0.f;
      const float* Li = Lp + pidx(i, 0);
      for (int j = lane; j < i; j += 32) part = fmaf(qb[j], Li[j], part);
      part = warp_sum(part);
      if (lane == 0) qb[i] = (qb[i] - part) * dinv[i];
      __syncwarp();
    }
    for (int i = lane; i < l; i += 32) Q[row * l + i] = qb[i];
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// One-sided Jacobi (Hestenes) SVD of an l x l matrix M, column-major.
// Round-robin (circle) ordering: l-1 rounds of l/2 disjoint column pairs per
// sweep; a pair (a, b) is rotated when |a.b| > tol sqrt(|a|^2 |b|^2), with
// the rotation that zeroes the new inner product.  V accumulates the
// rotations.  Stops after a sweep without rotations or after max_sweeps
// (then LRAMM_WARN_NOCONV is latched).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) jacobi_kernel(float* __restrict__ M, float* __restrict__ V,
                                                      int l, int max_sweeps, float tol, int* status) {
  __shared__ int s_rot;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int64_t e = tid; e < (int64_t)l * l; e += blockDim.x) V[e] = (e / l == e % l) ? 1.f : 0.f;
  const int n = (l + 1) & ~1;  // players; player l is a dummy when l is odd
  const int np = n / 2;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int t = 0; t < n - 1; ++t) {
      for (int kp = warp; kp < np; kp += nw) {
        int a, b;
        if (kp == 0) {
          a = 0;
          b = 1 + t % (n - 1);
        } else {
          a = 1 + (t + kp) % (n - 1);
          b = 1 + (t - kp + (n - 1)) % (n - 1);
        }
        if (a >= l || b >= l) continue;
        float* ca = M + (int64_t)a * l;
        float* cb = M + (int64_t)b * l;
        float al = 0.f, be = 0.f, ga = 0.f;
        for (int i = lane; i < l; i += 32) {
          const float x = ca[i], y = cb[i];
          al = fmaf(x, x, al);
          be = fmaf(y, y, be);
          ga = fmaf(x, y, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (!(fabsf(ga) > tol * sqrtf(al) * sqrtf(be))) continue;
        const float zeta = (be - al) / (2.0f * ga);
        float tt;
        if (fabsf(zeta) > 1e18f)
          tt = 0.5f / zeta;
        else
          tt = copysignf(1.0f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.0f)));
        const float c = 1.0f / sqrtf(fmaf(tt, tt, 1.0f));
        const float s = c * tt;
        // x' = c x - s y, y' = s x + c y applied as x - s (y + tau x) and
        // y + s (x - tau y), tau = s / (1 + c): for small angles fl(c) = 1
        // and the plain form would dilate both columns by 1 + t^2.
        const float tau = s / (1.0f + c);
        for (int i = lane; i < l; i += 32) {
          const float x = ca[i], y = cb[i];
          ca[i] = x - s * fmaf(tau, x, y);
          cb[i] = y + s * fmaf(-tau, y, x);
        }
        float* va = V + (int64_t)a * l;
        float* vb = V + (int64_t)b * l;
        for (int i = lane; i < l; i += 32) {
          const float x = va[i], y = vb[i];
          va[i] = x - s * fmaf(tau, x, y);
          vb[i] = y + s * fmaf(-tau, y, x);
        }
        if (lane == 0) s_rot = 1;
      }
      __syncthreads();
    }
    const int rot = s_rot;
    __syncthreads();
    if (!rot) break;
  }
  if (sweep >= max_sweeps && tid == 0) set_status(status, LRAMM_WARN_NOCONV);
}

// Sort columns by descending norm (sigma) and write the rank-r outputs.
__global__ void __launch_bounds__(1024) svd_finalize_kernel(const float* __restrict__ M,
                                                            const float* __restrict__ V, int l, int r,
                                                            float* __restrict__ sig,
                                                            float* __restrict__ S1, int s1_sigma,
                                                            float* __restrict__ S2, int s2_sigma) {
  extern __shared__ float sm[];
  float* nrm = sm;                               // l
  int* pos = reinterpret_cast<int*>(sm + l);     // l
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < l; j += nw) {
    float s = 0.f;
    for (int i = lane; i < l; i += 32) s = fmaf(M[(int64_t)j * l + i], M[(int64_t)j * l + i], s);
    s = warp_sum(s);
    if (lane == 0) nrm[j] = sqrtf(s);
  }
  __syncthreads();
  for (int j = tid; j < l; j += blockDim.x) {
    const float v = nrm[j];
    int rank = 0;
    for (int i = 0; i < l; ++i) {
      const float u = nrm[i];
      rank += (u > v) || (u == v && i < j);
    }
    pos[j] = rank;
  }
  __syncthreads();
  for (int j = warp; j < l; j += nw) {
    const int p = pos[j];
    if (p >= r) continue;
    const float sj = nrm[j];
    if (lane == 0) sig[p] = sj;
    const float u_scale = s1_sigma ? 1.0f : (sj > 0.f ? 1.0f / sj : 0.f);
    const float v_scale = s2_sigma ? sj : 1.0f;
    for (int i = lane; i < l; i += 32) {
      S1[(int64_t)i * r + p] = M[(int64_t)j * l + i] * u_scale;
      S2[(int64_t)i * r + p] = V[(int64_t)j * l + i] * v_scale;
    }
  }
}

// ---------------------------------------------------------------------------
// Opt-in shared memory per block on sm_100-class GPUs (227 KB), minus the
// static shared memory the kernels declare themselves.
static const int kSmemMax = 232448 - 1024;

lramm_status launch_chol(const float* G, int l, float shift_rel, float* L, int* status,
                         cudaStream_t s) {
  const size_t smem = sizeof(float) * (size_t)l * (l + 1) / 2;
  if (smem > (size_t)kSmemMax) return LRAMM_ERR_UNSUPPORTED;
  LRAMM_CUDA_TRY(cudaFuncSetAttribute(chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  chol_kernel<<<1, 1024, smem, s>>>(G, l, shift_rel, L, status);
  return last_launch();
}

lramm_status launch_trsm_rows(const float* Y, int64_t rows, int l, const float* L, float* Q,
                              cudaStream_t s) {
  const int threads = 1024, nw = threads / 32;
  const size_t smem = sizeof(float) * ((size_t)l * (l + 1) / 2 + l + (size_t)nw * l);
  if (smem > (size_t)kSmemMax) return LRAMM_ERR_UNSUPPORTED;
  LRAMM_CUDA_TRY(cudaFuncSetAttribute(trsm_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int64_t grid = ceil_div(rows, nw);
  if (grid > 152) grid = 152;
  trsm_rows_kernel<<<(unsigned)grid, threads, smem, s>>>(Y, rows, l, L, Q);
  return last_launch();
}

lramm_status launch_jacobi(float* M, float* V, int l, int max_sweeps, int* status, cudaStream_t s) {
  const float tol = 4.0f * sqrtf((float)l) * 0x1p-24f;
  jacobi_kernel<<<1, 1024, 0, s>>>(M, V, l, max_sweeps, tol, status);
  return last_launch();
}

lramm_status launch_svd_finalize(const float* M, const float* V, int l, int r, float* sig, float* S1,
                                 int s1_sigma, float* S2, int s2_sigma, cudaStream_t s) {
  const size_t smem = sizeof(float) * 2 * (size_t)l;
  svd_finalize_kernel<<<1, 1024, smem, s>>>(M, V, l, r, sig, S1, s1_sigma, S2, s2_sigma);
  return last_launch();
}

}  // namespace lramm
