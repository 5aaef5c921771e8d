// Orthonormalisation of the tall sketches by CholeskyQR (the "matrix Q with
// orthonormal columns" of the two-stage scheme, Sec. 2.2): for every problem
// of a batch (the A-side and B-side randomized SVDs run together)
//   G = Y^T Y                      gram_partial_kernel + gram_reduce_kernel
//   G + shift I = L L^T            chol2_kernel (one CTA per problem)
//   Q = Y L^-T                     trsm_panel_kernel (64 rows of Y per CTA)
// All FP32 with compensated or FP64 accumulation where sums are long.
#include <float.h>

#include "common.cuh"

namespace lramm {
namespace {

constexpr int kGT = 64;  // Gram tile

__device__ __forceinline__ float warp_max_o(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ int opidx(int i, int j) { return i * (i + 1) / 2 + j; }

// Lower-triangle tile t -> (ti, tj), tj <= ti.
__device__ __forceinline__ void tile_of(int t, int& ti, int& tj) {
  int r = static_cast<int>((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
  while (r * (r + 1) / 2 > t) --r;
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  ti = r;
  tj = t - r * (r + 1) / 2;
}

// Partial Gram of one lower 64 x 64 tile over a slice of rows: FP32 with
// 16-deep blocks added under Kahan compensation.
__global__ void __launch_bounds__(256)
gram_partial_kernel(GramBatch gb, int l, int ntiles, int splits, int64_t rows_per_split, float* __restrict__ part) {
  const GramProb& gp = gb.p[blockIdx.z];
  const float* __restrict__ Y = gp.Y;
  const int64_t rows = gp.rows;
  int ti, tj;
  tile_of(blockIdx.x, ti, tj);
  const int64_t k0 = static_cast<int64_t>(blockIdx.y) * rows_per_split;
  const int64_t k1 = min(rows, k0 + rows_per_split);
  const int m0 = ti * kGT, n0 = tj * kGT;
  __shared__ float As[16][kGT + 4];
  __shared__ float Bs[16][kGT + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4], cmp[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = cmp[i][j] = 0.f;
  for (int64_t kb = k0; kb < k1; kb += 16) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + u * 256;
      const int mm = e & 63, kk = e >> 6;
      const int64_t gk = kb + kk;
      As[kk][mm] = (gk < k1 && m0 + mm < l) ? Y[gk * l + m0 + mm] : 0.f;
      Bs[kk][mm] = (gk < k1 && n0 + mm < l) ? Y[gk * l + n0 + mm] : 0.f;
    }
    __syncthreads();
    float blk[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) blk[i][j] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) blk[i][j] = fmaf(a[i], b[j], blk[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float y = blk[i][j] - cmp[i][j];
        const float t = acc[i][j] + y;
        cmp[i][j] = (t - acc[i][j]) - y;
        acc[i][j] = t;
      }
    __syncthreads();
  }
  float* dst = part + ((static_cast<int64_t>(blockIdx.z) * splits + blockIdx.y) * ntiles + blockIdx.x) * kGT * kGT;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) dst[(ty * 4 + i) * kGT + tx * 4 + j] = acc[i][j];
}

// G[i][j] = sum over slices (FP64, fixed order) of the lower-tile partial
// holding (max(i,j), min(i,j)): symmetric by construction.
__global__ void gram_reduce_kernel(GramBatch gb, int l, int ntiles, int splits, const float* __restrict__ part) {
  const int64_t per = static_cast<int64_t>(l) * l;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < per * gb.n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int side = static_cast<int>(e / per);
    const int64_t rem = e - side * per;
    int i = static_cast<int>(rem / l), j = static_cast<int>(rem - static_cast<int64_t>(i) * l);
    const int a = i >= j ? i : j, b = i >= j ? j : i;
    const int ti = a / kGT, tj = b / kGT;
    const int tile = ti * (ti + 1) / 2 + tj;
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp)
      s += part[((static_cast<int64_t>(side) * splits + sp) * ntiles + tile) * kGT * kGT + (a % kGT) * kGT + (b % kGT)];
    gb.p[side].G[rem] = static_cast<float>(s);
  }
}

// Cholesky of G + shift_rel max(diag G) I, packed lower triangle in shared
// memory.  Columns are factored one at a time inside panels of 16 (thread 0
// takes the pivot and the panel part of the column, two barriers per
// column); after each panel the trailing matrix gets one rank-16 update in
// 4 x 4 register tiles.  A non-positive pivot latches LRAMM_ERR_NUMERIC and
// is replaced by a tiny positive value.
constexpr int kNB = 16;

__global__ void __launch_bounds__(1024) chol2_kernel(SmallBatch bt, int l, float shift_rel, int* status) {
  const float* __restrict__ G = bt.p[blockIdx.x].in;
  float* __restrict__ L = bt.p[blockIdx.x].out;
  extern __shared__ float P[];
  __shared__ float s_red[32];
  __shared__ float s_inv;
  __shared__ float s_col[kNB];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  float md = 0.f;
  for (int i = tid; i < l; i += blockDim.x) md = fmaxf(md, G[static_cast<int64_t>(i) * l + i]);
  md = warp_max_o(md);
  if (lane == 0) s_red[warp] = md;
  __syncthreads();
  if (warp == 0) {
    float v = lane < nw ? s_red[lane] : 0.f;
    v = warp_max_o(v);
    if (lane == 0) s_red[0] = v;
  }
  __syncthreads();
  const float shift = shift_rel * s_red[0];
  for (int i = warp; i < l; i += nw)
    for (int j = lane; j <= i; j += 32) P[opidx(i, j)] = G[static_cast<int64_t>(i) * l + j] + (i == j ? shift : 0.f);
  __syncthreads();

  for (int j0 = 0; j0 < l; j0 += kNB) {
    const int jend = min(j0 + kNB, l);
    for (int j = j0; j < jend; ++j) {
      if (tid == 0) {
        float d = P[opidx(j, j)];
        if (!(d > 0.f)) {
          set_status(status, LRAMM_ERR_NUMERIC);
          d = FLT_MIN * 1024.f;
        }
        d = sqrtf(d);
        P[opidx(j, j)] = d;
        const float inv = 1.0f / d;
        s_inv = inv;
        for (int c = j + 1; c < jend; ++c) s_col[c - j0] = P[opidx(c, j)] * inv;  // L[c][j], c in the panel
      }
      __syncthreads();
      const float inv = s_inv;
      for (int i = j + 1 + tid; i < l; i += blockDim.x) {
        const float lij = P[opidx(i, j)] * inv;
        P[opidx(i, j)] = lij;
        const int cend = min(jend - 1, i);
        for (int c = j + 1; c <= cend; ++c) P[opidx(i, c)] -= lij * s_col[c - j0];
      }
      __syncthreads();
    }
    // trailing update: rows i >= jend, columns c in [jend, i]
    const int n = l - jend;
    if (n > 0) {
      const int nb4 = (n + 3) / 4;
      const int ntile = nb4 * (nb4 + 1) / 2;
      for (int t = tid; t < ntile; t += blockDim.x) {
        int bi = static_cast<int>((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
        while (bi * (bi + 1) / 2 > t) --bi;
        while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
        const int bc = t - bi * (bi + 1) / 2;
        const int i0 = jend + 4 * bi, c0 = jend + 4 * bc;
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
        for (int k = j0; k < jend; ++k) {
          float a[4], b[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) a[u] = (i0 + u < l) ? P[opidx(i0 + u, k)] : 0.f;
#pragma unroll
          for (int v = 0; v < 4; ++v) b[v] = (c0 + v < l) ? P[opidx(c0 + v, k)] : 0.f;
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const int i = i0 + u, c = c0 + v;
            if (i < l && c <= i) P[opidx(i, c)] -= acc[u][v];
          }
      }
      __syncthreads();
    }
  }
  for (int64_t e = tid; e < static_cast<int64_t>(l) * l; e += blockDim.x) {
    const int i = static_cast<int>(e / l), j = static_cast<int>(e - static_cast<int64_t>(i) * l);
    L[e] = j <= i ? P[opidx(i, j)] : 0.f;
  }
}

// Q = Y L^-T for 64 rows of one problem per CTA: Q Lᵀ = Y is solved by
// 32-column panels, Q[:, J] = (Y[:, J] - Q[:, <J] L[J, <J]^T) L[J, J]^-T.
// The 64 rows live in shared memory; the panel of L is staged per step.
constexpr int kTR = 64, kTP = 32;

__global__ void __launch_bounds__(256) trsm_panel_kernel(SmallBatch bt, int l, int lq) {
  const SmallProb& sp = bt.p[blockIdx.y];
  const float* __restrict__ Y = sp.in;
  float* __restrict__ Q = sp.out;
  const float* __restrict__ L = sp.aux;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * kTR;
  if (r0 >= sp.rows) return;
  const int nrows = static_cast<int>(sp.rows - r0 < kTR ? sp.rows - r0 : kTR);
  extern __shared__ float sm[];
  float* Qs = sm;                            // kTR x lq
  float* Ls = Qs + kTR * lq;                 // kTP x (lq + 4): rows of L's panel
  float* Ld = Ls + kTP * (lq + 4);           // kTP x (kTP + 1): diagonal block
  const int tid = threadIdx.x;
  for (int e = tid; e < kTR * lq; e += blockDim.x) {
    const int r = e / lq, c = e - r * lq;
    Qs[e] = (r < nrows && c < l) ? Y[(r0 + r) * l + c] : 0.f;
  }
  const int np = (l + kTP - 1) / kTP;
  const int ls4 = lq + 4;
  for (int J = 0; J < np; ++J) {
    const int c0 = J * kTP;
    const int w = min(kTP, l - c0);
    // stage L[c0 .. c0+w, 0 .. c0+w)
    __syncthreads();
    for (int e = tid; e < kTP * (c0 + kTP); e += blockDim.x) {
      const int c = e / (c0 + kTP), k = e - c * (c0 + kTP);
      const float v = (c < w && k < c0 + w) ? L[static_cast<int64_t>(c0 + c) * l + k] : 0.f;
      if (k < c0)
        Ls[c * ls4 + k] = v;
      else
        Ld[c * (kTP + 1) + (k - c0)] = v;
    }
    __syncthreads();
    // update: thread (c, rows 8g..8g+7)
    if (c0 > 0) {
      const int c = tid & 31, g = tid >> 5;
      float acc[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] = 0.f;
      const float* lrow = Ls + c * ls4;
      for (int k = 0; k < c0; ++k) {
        const float b = lrow[k];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = fmaf(Qs[(8 * g + u) * lq + k], b, acc[u]);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) Qs[(8 * g + u) * lq + c0 + c] -= acc[u];
    }
    __syncthreads();
    // solve the 32-wide diagonal block row by row (one thread per row)
    if (tid < kTR) {
      float x[kTP];
      float* qrow = Qs + tid * lq + c0;
#pragma unroll
      for (int c = 0; c < kTP; ++c) {
        float v = qrow[c];
#pragma unroll
        for (int t = 0; t < c; ++t) v = fmaf(-x[t], Ld[c * (kTP + 1) + t], v);
        const float d = Ld[c * (kTP + 1) + c];
        x[c] = c < w ? v / d : 0.f;
      }
#pragma unroll
      for (int c = 0; c < kTP; ++c) qrow[c] = x[c];
    }
  }
  __syncthreads();
  for (int e = tid; e < nrows * l; e += blockDim.x) {
    const int r = e / l, c = e - r * l;
    Q[(r0 + r) * l + c] = Qs[r * lq + c];
  }
}

}  // namespace

size_t gram_part_floats(int l) {
  // splits * tiles <= ~2 * 152 per problem, two problems
  (void)l;
  return static_cast<size_t>(2) * 320 * kGT * kGT;
}

lramm_status launch_gram(GramBatch gb, int l, float* part, cudaStream_t s) {
  const int nt = (l + kGT - 1) / kGT;
  const int ntiles = nt * (nt + 1) / 2;
  int64_t rows = 0;
  for (int i = 0; i < gb.n; ++i) rows = gb.p[i].rows > rows ? gb.p[i].rows : rows;
  int splits = static_cast<int>((2 * 152 + ntiles - 1) / ntiles);
  if (splits > 320 / ntiles) splits = 320 / ntiles;
  if (splits < 1) splits = 1;
  int64_t rps = ceil_div(ceil_div(rows, splits), 16) * 16;
  if (rps < 64) rps = 64;
  splits = static_cast<int>(ceil_div(rows, rps));
  if (static_cast<size_t>(gb.n) * splits * ntiles > 2 * 320) return LRAMM_ERR_UNSUPPORTED;
  gram_partial_kernel<<<dim3(ntiles, splits, gb.n), 256, 0, s>>>(gb, l, ntiles, splits, rps, part);
  LRAMM_TRY(last_launch());
  int64_t g = ceil_div(static_cast<int64_t>(l) * l * gb.n, 256);
  if (g > 152 * 8) g = 152 * 8;
  gram_reduce_kernel<<<static_cast<unsigned>(g), 256, 0, s>>>(gb, l, ntiles, splits, part);
  return last_launch();
}

static const int kSmemMaxO = 232448 - 1024;

lramm_status launch_chol2(SmallBatch bt, int l, float shift_rel, int* status, cudaStream_t s) {
  const size_t smem = sizeof(float) * static_cast<size_t>(l) * (l + 1) / 2;
  if (smem > static_cast<size_t>(kSmemMaxO)) return LRAMM_ERR_UNSUPPORTED;
  LRAMM_CUDA_TRY(cudaFuncSetAttribute(chol2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  chol2_kernel<<<bt.n, 1024, smem, s>>>(bt, l, shift_rel, status);
  return last_launch();
}

lramm_status launch_trsm_panel(SmallBatch bt, int l, cudaStream_t s) {
  const int lq = static_cast<int>(round_up(l, kTP)) + 1;
  const size_t smem = sizeof(float) * (static_cast<size_t>(kTR) * lq + static_cast<size_t>(kTP) * (lq + 4) +
                                       static_cast<size_t>(kTP) * (kTP + 1));
  if (smem > static_cast<size_t>(kSmemMaxO)) return LRAMM_ERR_UNSUPPORTED;
  LRAMM_CUDA_TRY(
      cudaFuncSetAttribute(trsm_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
  int64_t rows = 0;
  for (int i = 0; i < bt.n; ++i) rows = bt.p[i].rows > rows ? bt.p[i].rows : rows;
  trsm_panel_kernel<<<dim3(static_cast<unsigned>(ceil_div(rows, kTR)), bt.n), 256, smem, s>>>(bt, l, lq);
  return last_launch();
}

}  // namespace lramm
