// Orthonormalisation of the tall sketches by CholeskyQR (the "matrix Q with
// orthonormal columns" of the two-stage scheme, Sec. 2.2): for every problem
// of a batch (the A-side and B-side randomized SVDs run together)
//   G = Y^T Y                      gram_partial_kernel + gram_reduce_kernel
//   G + shift I = L L^T            chol2_kernel (one CTA per problem)
//   Q = Y L^-T                     trsm_panel_kernel (64 rows of Y per CTA)
// All FP32 with compensated or FP64 accumulation where sums are long.
#include <float.h>

#include "common.cuh"
#include "tc_common.cuh"

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
// 16-deep blocks added under Kahan compensation.  Rows arrive through a
// register-prefetched double buffer (one barrier per 16 rows); every thread
// owns a 4 x 4 block and reads its operands as float4 broadcasts.  VEC: rows
// of Y are 16-byte aligned (l % 4 == 0), one float4 per thread and operand.
template <bool VEC>
__global__ void __launch_bounds__(256)
gram_partial_kernel(GramBatch gb, int l, int ntiles, int splits, int64_t rows_per_split, float* __restrict__ part,
                    const int* __restrict__ cond) {
  if (cond && *cond == 0) return;
  const GramProb& gp = gb.p[blockIdx.z];
  const float* __restrict__ Y = gp.Y;
  const int64_t rows = gp.rows;
  int ti, tj;
  tile_of(blockIdx.x, ti, tj);
  const int64_t k0 = static_cast<int64_t>(blockIdx.y) * rows_per_split;
  const int64_t k1 = min(rows, k0 + rows_per_split);
  const int m0 = ti * kGT, n0 = tj * kGT;
  __shared__ __align__(16) float As[2][16][kGT];
  __shared__ __align__(16) float Bs[2][16][kGT];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int lk = tid >> 4, lc = (tid & 15) * 4;   // loader: row lk, columns lc .. lc+3
  float acc[4][4], cmp[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = cmp[i][j] = 0.f;
  float4 ra, rb;
  auto fetch = [&](int64_t kb) {
    const int64_t gk = kb + lk;
    const float* yr = Y + gk * l;
    const bool rok = gk < k1;
    if (VEC) {
      ra = (rok && m0 + lc < l) ? *reinterpret_cast<const float4*>(yr + m0 + lc) : make_float4(0.f, 0.f, 0.f, 0.f);
      rb = (rok && n0 + lc < l) ? *reinterpret_cast<const float4*>(yr + n0 + lc) : make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      ra.x = (rok && m0 + lc + 0 < l) ? yr[m0 + lc + 0] : 0.f;
      ra.y = (rok && m0 + lc + 1 < l) ? yr[m0 + lc + 1] : 0.f;
      ra.z = (rok && m0 + lc + 2 < l) ? yr[m0 + lc + 2] : 0.f;
      ra.w = (rok && m0 + lc + 3 < l) ? yr[m0 + lc + 3] : 0.f;
      rb.x = (rok && n0 + lc + 0 < l) ? yr[n0 + lc + 0] : 0.f;
      rb.y = (rok && n0 + lc + 1 < l) ? yr[n0 + lc + 1] : 0.f;
      rb.z = (rok && n0 + lc + 2 < l) ? yr[n0 + lc + 2] : 0.f;
      rb.w = (rok && n0 + lc + 3 < l) ? yr[n0 + lc + 3] : 0.f;
    }
  };
  if (k0 < k1) {
    fetch(k0);
    *reinterpret_cast<float4*>(&As[0][lk][lc]) = ra;
    *reinterpret_cast<float4*>(&Bs[0][lk][lc]) = rb;
  }
  __syncthreads();
  int cur = 0;
  for (int64_t kb = k0; kb < k1; kb += 16) {
    const bool more = kb + 16 < k1;
    if (more) fetch(kb + 16);
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
      for (int j = 0; j < 4; ++j) {
        const float y = blk[i][j] - cmp[i][j];
        const float t = acc[i][j] + y;
        cmp[i][j] = (t - acc[i][j]) - y;
        acc[i][j] = t;
      }
    if (more) {
      *reinterpret_cast<float4*>(&As[cur ^ 1][lk][lc]) = ra;
      *reinterpret_cast<float4*>(&Bs[cur ^ 1][lk][lc]) = rb;
    }
    __syncthreads();
    cur ^= 1;
  }
  float* dst = part + ((static_cast<int64_t>(blockIdx.z) * splits + blockIdx.y) * ntiles + blockIdx.x) * kGT * kGT;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    *reinterpret_cast<float4*>(dst + (ty * 4 + i) * kGT + tx * 4) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
}

// Partial Gram of one lower 64 x 64 tile over a slice of rows, 64 threads
// each owning an 8 x 8 block -- rows {4ty..4ty+3, 32+4ty..32+4ty+3} x the
// same split of columns by tx, so that each float4 read of a warp covers one
// contiguous 64- or 128-byte span (no bank conflicts): four float4 reads
// feed 64 FMAs.
// Rows arrive through a register-prefetched double buffer (8 float4 global
// loads per thread per 16 rows).  Plain FP32 FMA chains over the slice (a
// few hundred rows); the slices are added in FP64 by the reduction.
// Needs l % 4 == 0 and 16-byte aligned rows.
__global__ void __launch_bounds__(64)
gram_partial8_kernel(GramBatch gb, int l, int ntiles, int splits, int64_t rows_per_split, float* __restrict__ part,
                     const int* __restrict__ cond) {
  if (cond && *cond == 0) return;
  const GramProb& gp = gb.p[blockIdx.z];
  const float* __restrict__ Y = gp.Y;
  const int64_t rows = gp.rows;
  int ti, tj;
  tile_of(blockIdx.x, ti, tj);
  const int64_t k0 = static_cast<int64_t>(blockIdx.y) * rows_per_split;
  const int64_t k1 = min(rows, k0 + rows_per_split);
  const int m0 = ti * kGT, n0 = tj * kGT;
  __shared__ __align__(16) float As[2][16][kGT];
  __shared__ __align__(16) float Bs[2][16][kGT];
  const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  // loader: 16 rows x 16 float4 per operand = 256 float4 = 4 per thread
  float4 ra[4], rb[4];
  auto fetch = [&](int64_t kb) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int q = tid + 64 * u, kk = q >> 4, c4 = (q & 15) * 4;
      const int64_t gk = kb + kk;
      const float* yr = Y + gk * l;
      const bool rok = gk < k1;
      ra[u] = (rok && m0 + c4 < l) ? *reinterpret_cast<const float4*>(yr + m0 + c4) : make_float4(0.f, 0.f, 0.f, 0.f);
      rb[u] = (rok && n0 + c4 < l) ? *reinterpret_cast<const float4*>(yr + n0 + c4) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int q = tid + 64 * u, kk = q >> 4, c4 = (q & 15) * 4;
      *reinterpret_cast<float4*>(&As[buf][kk][c4]) = ra[u];
      *reinterpret_cast<float4*>(&Bs[buf][kk][c4]) = rb[u];
    }
  };
  if (k0 < k1) {
    fetch(k0);
    stash(0);
  }
  __syncthreads();
  int cur = 0;
  for (int64_t kb = k0; kb < k1; kb += 16) {
    const bool more = kb + 16 < k1;
    if (more) fetch(kb + 16);
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][kk][32 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][kk][32 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) stash(cur ^ 1);
    __syncthreads();
    cur ^= 1;
  }
  float* dst = part + ((static_cast<int64_t>(blockIdx.z) * splits + blockIdx.y) * ntiles + blockIdx.x) * kGT * kGT;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float* rowp = dst + (i < 4 ? ty * 4 + i : 32 + ty * 4 + i - 4) * kGT;
    *reinterpret_cast<float4*>(rowp + tx * 4) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    *reinterpret_cast<float4*>(rowp + 32 + tx * 4) = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
  }
}

// G = sum over slices of the lower-tile partials, in slice order with Kahan
// compensation (FP32; error ~2u of the sum of magnitudes); the transposed
// entry of an off-diagonal tile is written from the same sum, and a diagonal
// tile holds both triangles computed from identical products, so G is
// exactly symmetric.  Each thread adds four consecutive elements of a tile
// row (float4 reads of the partials, four slices in flight).
__global__ void gram_reduce_kernel(GramBatch gb, int l, int ntiles, int splits, const float* __restrict__ part,
                                   const int* __restrict__ cond) {
  if (cond && *cond == 0) return;
  const int64_t per4 = static_cast<int64_t>(ntiles) * kGT * kGT / 4;
  const int64_t tile_stride4 = per4;   // between slices
  const float4* part4 = reinterpret_cast<const float4*>(part);
  for (int64_t e4 = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e4 < per4 * gb.n;
       e4 += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int side = static_cast<int>(e4 / per4);
    const int64_t rem4 = e4 - side * per4;
    const int tile = static_cast<int>(rem4 >> 10), idx = static_cast<int>(rem4 & 1023) * 4;
    int ti, tj;
    tile_of(tile, ti, tj);
    const int i = ti * kGT + (idx >> 6), j = tj * kGT + (idx & 63);
    if (i >= l || j >= l) continue;
    const float4* src = part4 + static_cast<int64_t>(side) * splits * tile_stride4 + rem4;
    float sum[4] = {0.f, 0.f, 0.f, 0.f}, cmp[4] = {0.f, 0.f, 0.f, 0.f};
    auto add = [&](const float4& v) {
      const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float y = x[t] - cmp[t];
        const float u = sum[t] + y;
        cmp[t] = (u - sum[t]) - y;
        sum[t] = u;
      }
    };
    int sp = 0;
    for (; sp + 4 <= splits; sp += 4) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = src[static_cast<int64_t>(sp + u) * tile_stride4];
#pragma unroll
      for (int u = 0; u < 4; ++u) add(v[u]);
    }
    for (; sp < splits; ++sp) add(src[static_cast<int64_t>(sp) * tile_stride4]);
    float* G = gb.p[side].G;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (j + t >= l) break;
      G[static_cast<int64_t>(i) * l + j + t] = sum[t];
      if (ti != tj) G[static_cast<int64_t>(j + t) * l + i] = sum[t];
    }
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

// ---------------------------------------------------------------------------
// Blocked Cholesky with 32-column panels (one CTA per problem, 512 threads,
// packed lower triangle in shared memory).  Per panel J:
//   (a) warp 0 factors the 32 x 32 diagonal block in registers: lane i holds
//       row i, pivots and columns travel by shuffles (no CTA barrier inside);
//   (b) one thread per row below solves L_IJ L_JJ^T = A_IJ in registers by
//       forward substitution, reading columns of L_JJ as float4 broadcasts;
//   (c) the trailing update A_22 -= L_2J L_2J^T in 4 x 4 register tiles from
//       a transposed copy of the panel.
// While warp 0 factors diagonal block J+1, four warps write column block J
// of L to global memory and, when the problem asks for them (Xd given: the
// panel triangular solve), eight warps invert L_JJ, all on the SM
// sub-partitions other than warp 0's; the last block follows the panel loop.
// A non-positive pivot latches LRAMM_ERR_NUMERIC and is replaced by a tiny
// positive value, as in chol2_kernel.
// ---------------------------------------------------------------------------
constexpr int kCB = 32;
constexpr int kLC = kCB + 4;   // row stride of the column-major copy of L_JJ

__host__ __device__ inline int chol_split_h_dev(int l) {
  const int h = ((l + 1) / 2 + kCB - 1) / kCB * kCB;
  return h < 288 ? h : 288;
}

// Inverse of the diagonal block at j0 (w x w, w <= 32) of the packed
// factor P into xg (32 x 32 row-major, zero outside w x w), by the eight
// warps v = 0..7 of the calling group (named barrier 2, 256 threads): column
// c = 4v + lane / 8 on the eight lanes 8 (lane / 8) .. +7, lane e of them
// holding rows e, e+8, e+16, e+24.  Forward substitution in column order
// (b = e_c; for each t: x_t = b_t / L_tt, then b_i -= L_it x_t for i > t;
// finally x_i = b_i / L_ii): each x_i is the same FP32 chain as the
// row-order substitution x_i = -(sum_t L_it x_t) / L_ii.  s_rl: 32 floats.
__device__ __forceinline__ void chol_inv_block(const float* P, int j0, int w, float* xg, float* s_rl, int v,
                                               int lane) {
  if (v == 0) s_rl[lane] = 1.0f / (lane < w ? P[opidx(j0 + lane, j0 + lane)] : 1.0f);
  asm volatile("bar.sync 2, 256;" ::: "memory");
  const int c = 4 * v + (lane >> 3), e = lane & 7, base = lane & ~7;
  float b[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) b[u] = e + 8 * u == c ? 1.f : 0.f;
#pragma unroll 1
  for (int t = 0; t < w; ++t) {
    // b_t from its owner lane (slot t / 8, picked with bit masks: a
    // conditional pick was turned into a local-memory copy of b)
    const uint32_t su = static_cast<uint32_t>(t >> 3);
    uint32_t mine = 0u;
#pragma unroll
    for (int u = 0; u < 4; ++u) mine |= __float_as_uint(b[u]) & (0u - static_cast<uint32_t>(su == u));
    const float xt = __uint_as_float(__shfl_sync(0xffffffffu, mine, base | (t & 7))) * s_rl[t];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = e + 8 * u;
      if (i > t && i < w) b[u] = fmaf(-P[opidx(j0 + i, j0 + t)], xt, b[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = e + 8 * u;
    xg[i * kCB + c] = (i < w && c < w) ? b[u] * s_rl[i] : 0.f;
  }
}

// The eight inverting warps of chol3_kernel: 1, 2, 3, 5, 6, 7, 9, 10 (none
// on warp 0's SM sub-partition), numbered 0..7.
__device__ __forceinline__ bool inv_warp(int w) { return (w & 3) != 0 && w <= 10; }
__device__ __forceinline__ int inv_index(int w) { return w - 1 - (w > 4) - (w > 8); }

// Column block j0 .. j0+31 of L (row-major, zero above the diagonal) from
// the packed factor, rows v, v + nv, ..; lane = column.
__device__ __forceinline__ void chol_write_L_block(const float* P, float* Lo, int l, int j0, int v, int nv, int lane) {
  const int col = j0 + lane;
  if (col >= l) return;
  for (int r = v; r < l; r += nv) Lo[static_cast<int64_t>(r) * l + col] = r >= col ? P[opidx(r, col)] : 0.f;
}

// TC: the trailing update runs on the tensor cores (kind::tf32, split into
// TF32 high and low parts: hi hi + lo hi + hi lo, FP32 accumulation in TMEM)
// from two 128-byte-swizzled K-major copies of the panel below the diagonal
// block (256 rows x 32 columns each); otherwise in FP32 SIMT register tiles.
template <bool TC>
__global__ void __launch_bounds__(512, 1) chol3_kernel(CholBatch cb, int l, float shift_rel, float shift_big_rel,
                                                       int* status, const int* __restrict__ cond) {
  if (cond && *cond == 0) return;   // predicated launch (the CholeskyQR fallback)
  const CholProb& cp = cb.p[blockIdx.x];
  const float* __restrict__ G = cp.G;
  float* __restrict__ Lo = cp.L;
  float* __restrict__ Xd = cp.Xd;
  extern __shared__ float4 c3_smem4[];
  float* P = reinterpret_cast<float*>(c3_smem4);
  const int np = l * (l + 1) / 2;
  const int lp = static_cast<int>(round_up(l, 4)) + 4;   // row stride of the transposed panel
  // Row j of the trailing block sits at position ((j & 4) ? H : 0) + 4 (j >> 3) + (j & 3)
  // of a panel row: the halves of each 8-row group in two regions, so that
  // both the 4-row and the 8-row tiles of the update read them as float4
  // runs at a 16-byte stride across threads (no bank conflict).
  const int H = 4 * ((l + 7) / 8);
  float* PnT = P + round_up(np, 4);                       // kCB x lp (SIMT update)
  float* LC = TC ? PnT : PnT + kCB * lp;                  // kCB x kLC: LC[t][c] = L_JJ[c][t], c > t
  __shared__ float s_red[32];
  __shared__ float s_rinv[kCB];
  __shared__ float s_rl[kCB];   // 1 / L_tt of the diagonal block being inverted
  __shared__ __align__(16) float s_dcol[2 * kCB];   // the current pivot's column, two buffers
  __shared__ int s_bad;   // a pivot of this attempt was not positive
  __shared__ __align__(8) uint64_t s_mbar;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  // TC: panel copies at the first 1024-byte boundary after LC (hi: 32 KB, lo: 32 KB)
  uint8_t* T_hi = nullptr;
  uint8_t* T_lo = nullptr;
  uint32_t mphase = 0;
  // TMEM: one 128-column accumulator while the trailing block has at most
  // 128 rows (l <= 160), else two tiles at columns 0 and 256 (kept small so
  // that the CTA finds room beside other kernels' accumulators on its SM)
  const uint32_t tmem_cols = l - kCB <= 128 ? 128u : 512u;
  if (TC) {
    uint8_t* after = reinterpret_cast<uint8_t*>(LC + kCB * kLC);
    T_hi = after + ((1024u - (tc::smem_u32(after) & 1023u)) & 1023u);
    T_lo = T_hi + 256 * 128;
    if (tid == 0) {
      tc::mbar_init(&s_mbar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&s_tmem)),
                   "r"(tmem_cols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
  }
  if (tid == 0) s_bad = 0;
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
  // Attempt 0 factors G + shift_rel max(diag) I.  If a pivot is not positive
  // and shift_big_rel > 0, attempt 1 factors G + shift_big_rel max(diag) I
  // from scratch (the shifted CholeskyQR fallback: the caller then adds a
  // pass).  A non-positive pivot of the last attempt is replaced by a tiny
  // positive value and reported.
  bool restarted = false;
  for (int attempt = 0;; ++attempt) {
    const float shift = (attempt == 0 ? shift_rel : shift_big_rel) * s_red[0];
    {  // G (row-major, l % 4 == 0) into the packed lower triangle: 8 float4 loads in flight per thread
      const int nq = l * l / 4, lq4 = l / 4;
      const float4* G4 = reinterpret_cast<const float4*>(G);
      for (int q0 = tid; q0 < nq; q0 += 8 * blockDim.x) {
        float4 v[8];
  #pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int q = q0 + u * blockDim.x;
          if (q < nq) v[u] = G4[q];
        }
  #pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int q = q0 + u * blockDim.x;
          if (q >= nq) break;
          const int i = q / lq4, j = 4 * (q - i * lq4);
          const float e4[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
  #pragma unroll
          for (int t = 0; t < 4; ++t)
            if (j + t <= i) P[opidx(i, j + t)] = e4[t] + (i == j + t ? shift : 0.f);
        }
      }
    }
    if (!TC)
      for (int e = tid; e < kCB * lp; e += blockDim.x) PnT[e] = 0.f;
    __syncthreads();

    for (int j0 = 0; j0 < l; j0 += kCB) {
      const int w = min(kCB, l - j0);
      if (warp == 0) {
        float a[kCB];
  #pragma unroll
        for (int c = 0; c < kCB; ++c)
          a[c] = lane < w ? (c <= lane ? P[opidx(j0 + lane, j0 + c)] : 0.f) : (c == lane ? 1.f : 0.f);
        // The pivot chain is software-pipelined: lane k+1 forms its own next
        // diagonal entry from its own multiplier (the value the shuffled update
        // below gives it, bit for bit), and that entry is broadcast before the
        // remaining updates of this pivot issue.  A non-positive pivot is
        // replaced without a branch and latched once after the block, so the
        // unrolled pivots form straight-line code.
        // The column l_ck of each pivot reaches the lanes through shared
        // memory (one store a lane, float4 broadcast reads, two buffers so
        // that one __syncwarp a pivot suffices) instead of a shuffle per
        // column: the same FMAs in the same order.
        bool bad = false;
        float piv = __shfl_sync(0xffffffffu, a[0], 0);
  #pragma unroll
        for (int k = 0; k < kCB; ++k) {
          bad |= !(piv > 0.f);
          piv = piv > 0.f ? piv : FLT_MIN * 1024.f;
          const float inv = rsqrtf(piv);
          const float lk = lane == k ? piv * inv : a[k] * inv;
          a[k] = lk;
          if (lane == k) s_rinv[k] = inv;
          float piv_next = 0.f;
          if (k + 1 < kCB) piv_next = __shfl_sync(0xffffffffu, fmaf(-lk, lk, a[k + 1]), k + 1);
          float* dcol = s_dcol + (k & 1) * kCB;
          dcol[lane] = lk;
          __syncwarp();
  #pragma unroll
          for (int c4 = ((k + 1) / 4) * 4; c4 < kCB; c4 += 4) {
            const float4 v = *reinterpret_cast<const float4*>(dcol + c4);
            if (c4 + 0 > k) a[c4 + 0] = fmaf(-lk, v.x, a[c4 + 0]);
            if (c4 + 1 > k) a[c4 + 1] = fmaf(-lk, v.y, a[c4 + 1]);
            if (c4 + 2 > k) a[c4 + 2] = fmaf(-lk, v.z, a[c4 + 2]);
            if (c4 + 3 > k) a[c4 + 3] = fmaf(-lk, v.w, a[c4 + 3]);
          }
          piv = piv_next;
        }
        if (bad && lane == 0) s_bad = 1;
  #pragma unroll
        for (int c = 0; c < kCB; ++c) {
          if (lane < w && c <= lane) P[opidx(j0 + lane, j0 + c)] = a[c];
          LC[c * kLC + lane] = (lane < w && c < lane) ? a[c] : 0.f;
        }
      } else if (j0 > 0) {
        // meanwhile the previous column block is final: eight warps invert
        // its diagonal block and four write it to L, all on the three SM
        // sub-partitions that do not issue warp 0 (warps 4, 8, 12 idle)
        if (Xd != nullptr && inv_warp(warp))
          chol_inv_block(P, j0 - kCB, kCB, Xd + static_cast<int64_t>(j0 / kCB - 1) * kCB * kCB, s_rl,
                         inv_index(warp), lane);
        else if (nw == 16 && (warp == 11 || warp >= 13))
          chol_write_L_block(P, Lo, l, j0 - kCB, warp == 11 ? 0 : warp - 12, 4, lane);
        else if (nw < 16 && (warp & 3) != 0)   // fewer threads (no inversion): warps off warp 0's sub-partition
          chol_write_L_block(P, Lo, l, j0 - kCB, warp - 1 - (warp >> 2), 3 * nw / 4, lane);
      }
      __syncthreads();
      const int r0 = j0 + kCB;   // first row below the diagonal block
      const int n2 = l - r0;
      if (n2 <= 0) break;
      // (b) rows below: x L_JJ^T = a, right-looking in registers
      if (tid < n2) {
        const int row = r0 + tid;
        float a[kCB];
  #pragma unroll
        for (int t = 0; t < kCB; ++t) a[t] = P[opidx(row, j0 + t)];
  #pragma unroll
        for (int t = 0; t < kCB; ++t) {
          const float x = a[t] * s_rinv[t];
          a[t] = x;
  #pragma unroll
          for (int c4 = ((t + 1) / 4) * 4; c4 < kCB; c4 += 4) {
            const float4 lv = *reinterpret_cast<const float4*>(LC + t * kLC + c4);
            if (c4 + 0 > t) a[c4 + 0] = fmaf(-x, lv.x, a[c4 + 0]);
            if (c4 + 1 > t) a[c4 + 1] = fmaf(-x, lv.y, a[c4 + 1]);
            if (c4 + 2 > t) a[c4 + 2] = fmaf(-x, lv.z, a[c4 + 2]);
            if (c4 + 3 > t) a[c4 + 3] = fmaf(-x, lv.w, a[c4 + 3]);
          }
        }
  #pragma unroll
        for (int t = 0; t < kCB; ++t) P[opidx(row, j0 + t)] = a[t];
        if (TC) {  // row tid of the swizzled copies: 16-byte chunk c at position c ^ (tid mod 8)
          uint8_t* hr = T_hi + tid * 128;
          uint8_t* lr = T_lo + tid * 128;
  #pragma unroll
          for (int c = 0; c < kCB / 4; ++c) {
            float h[4], o[4];
  #pragma unroll
            for (int e = 0; e < 4; ++e) {
              h[e] = __uint_as_float(__float_as_uint(a[4 * c + e]) & 0xFFFFE000u);
              o[e] = a[4 * c + e] - h[e];
            }
            const int off = (c ^ (tid & 7)) * 16;
            *reinterpret_cast<float4*>(hr + off) = make_float4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<float4*>(lr + off) = make_float4(o[0], o[1], o[2], o[3]);
          }
        } else {
          const int pos = ((tid & 4) ? H : 0) + 4 * (tid >> 3) + (tid & 3);
  #pragma unroll
          for (int t = 0; t < kCB; ++t) PnT[t * lp + pos] = a[t];
        }
      }
      __syncthreads();
      // (c) trailing update, rows/cols r0 .. l-1, lower triangle
      if (TC) {
        // D_t = rows 128 t .. 128 t + 127 of the panel copy times the first N_t
        // rows (only columns c <= i are needed); TMEM columns 256 t ..
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        const int N = static_cast<int>(round_up(n2, 32));
        const int tiles = (n2 + 127) / 128;
        const uint32_t tm = s_tmem;
        if (tid == 0) {
          tc::tc_fence_after();
          for (int t = 0; t < tiles; ++t) {
            const int Nt = t == 0 ? min(N, 128) : N;
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(Nt >> 3) << 17) |
                                   (static_cast<uint32_t>(128 >> 4) << 24);
            const uint32_t ah = tc::smem_u32(T_hi + t * 16384), al = tc::smem_u32(T_lo + t * 16384);
            const uint32_t bh = tc::smem_u32(T_hi), bl = tc::smem_u32(T_lo);
  #pragma unroll
            for (int kk = 0; kk < 4; ++kk) {   // 8 TF32 (32 bytes) of K per instruction
              const uint64_t dah = tc::kmajor_sw128_desc(ah + kk * 32), dal = tc::kmajor_sw128_desc(al + kk * 32);
              const uint64_t dbh = tc::kmajor_sw128_desc(bh + kk * 32), dbl = tc::kmajor_sw128_desc(bl + kk * 32);
              const uint32_t d = tm + static_cast<uint32_t>(t * 256);
              asm volatile(
                  "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                  "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                  "l"(dah), "l"(dbh), "r"(idesc), "r"(kk > 0 ? 1u : 0u)
                  : "memory");
              asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;" ::"r"(d), "l"(dal), "l"(dbh),
                           "r"(idesc)
                           : "memory");
              asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;" ::"r"(d), "l"(dah), "l"(dbl),
                           "r"(idesc)
                           : "memory");
            }
          }
          tc::mma_commit(&s_mbar);
        }
        volatile int never = 0;
        if (!tc::mbar_wait(&s_mbar, mphase, &never) && tid == 0) set_status(status, LRAMM_ERR_TIMEOUT);
        mphase ^= 1u;
        tc::tc_fence_after();
        const int q = warp & 3, part = warp >> 2;   // TMEM lanes 32 q .. 32 q + 31; column chunks part, part + nw / 4
        for (int t = 0; t < tiles; ++t) {
          const int Nt = t == 0 ? min(N, 128) : N;
          for (int ch = part; ch < Nt / 32; ch += nw >> 2) {
            float v[32];
            tc::tmem_ld32(tm + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(t * 256 + ch * 32), v);
            const int j = t * 128 + q * 32 + lane;
            const int i = r0 + j;
            if (j < n2) {
  #pragma unroll
              for (int jj = 0; jj < 32; ++jj) {
                const int c = r0 + ch * 32 + jj;
                if (c <= i) P[opidx(i, c)] -= v[jj];
              }
            }
          }
        }
        tc::tc_fence_before();
      } else if (n2 >= 96) {  // 8 x 8 tiles
        const int nb8 = (n2 + 7) / 8;
        const int ntile = nb8 * (nb8 + 1) / 2;
        for (int t = tid; t < ntile; t += blockDim.x) {
          int bi = static_cast<int>((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
          while (bi * (bi + 1) / 2 > t) --bi;
          while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
          const int bc = t - bi * (bi + 1) / 2;
          float acc[8][8];
  #pragma unroll
          for (int u = 0; u < 8; ++u)
  #pragma unroll
            for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;
  #pragma unroll 1
          for (int k = 0; k < kCB; ++k) {
            const float* row = PnT + k * lp;
            const float4 a0 = *reinterpret_cast<const float4*>(row + 4 * bi);
            const float4 a1 = *reinterpret_cast<const float4*>(row + H + 4 * bi);
            const float4 b0 = *reinterpret_cast<const float4*>(row + 4 * bc);
            const float4 b1 = *reinterpret_cast<const float4*>(row + H + 4 * bc);
            const float a8[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b8[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
  #pragma unroll
            for (int u = 0; u < 8; ++u)
  #pragma unroll
              for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(a8[u], b8[v], acc[u][v]);
          }
  #pragma unroll
          for (int u = 0; u < 8; ++u)
  #pragma unroll
            for (int v = 0; v < 8; ++v) {
              const int i = r0 + 8 * bi + u, c = r0 + 8 * bc + v;
              if (i < l && c <= i) P[opidx(i, c)] -= acc[u][v];
            }
        }
      } else {  // 4 x 4 tiles
        const int nb4 = (n2 + 3) / 4;
        const int ntile = nb4 * (nb4 + 1) / 2;
        for (int t = tid; t < ntile; t += blockDim.x) {
          int bi = static_cast<int>((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
          while (bi * (bi + 1) / 2 > t) --bi;
          while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
          const int bc = t - bi * (bi + 1) / 2;
          float acc[4][4];
  #pragma unroll
          for (int u = 0; u < 4; ++u)
  #pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
  #pragma unroll 8
          for (int k = 0; k < kCB; ++k) {
            const float4 av = *reinterpret_cast<const float4*>(PnT + k * lp + ((bi & 1) ? H : 0) + 4 * (bi >> 1));
            const float4 bv = *reinterpret_cast<const float4*>(PnT + k * lp + ((bc & 1) ? H : 0) + 4 * (bc >> 1));
            const float a4[4] = {av.x, av.y, av.z, av.w};
            const float b4[4] = {bv.x, bv.y, bv.z, bv.w};
  #pragma unroll
            for (int u = 0; u < 4; ++u)
  #pragma unroll
              for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a4[u], b4[v], acc[u][v]);
          }
  #pragma unroll
          for (int u = 0; u < 4; ++u)
  #pragma unroll
            for (int v = 0; v < 4; ++v) {
              const int i = r0 + 4 * bi + u, c = r0 + 4 * bc + v;
              if (i < l && c <= i) P[opidx(i, c)] -= acc[u][v];
            }
        }
      }
      __syncthreads();
    }
    __syncthreads();
    if (!s_bad || attempt > 0 || !(shift_big_rel > 0.f)) break;
    __syncthreads();   // every thread has read s_bad
    if (tid == 0) s_bad = 0;
    restarted = true;
  }
  if (tid == 0) {
    if (s_bad) {
      if (cp.brk) {   // the caller retries with a larger shift
        *cp.brk = 1;
        if (cp.brk_any) *cp.brk_any = 1;
      } else {
        set_status(status, LRAMM_ERR_NUMERIC);
      }
    }
    if (restarted && cp.brk_any) *cp.brk_any = 1;
    if ((restarted || s_bad) && cp.brk_count) atomicAdd(cp.brk_count, 1);
  }
  if (TC && warp == 1) {
    tc::tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem), "r"(tmem_cols) : "memory");
  }
  // The last column block (the others were written and inverted inside the
  // panel loop, during the next diagonal block's factorisation).
  {
    const int jl = ((l - 1) / kCB) * kCB;
    if (Xd == nullptr)
      chol_write_L_block(P, Lo, l, jl, warp, nw, lane);
    else if (inv_warp(warp))
      chol_inv_block(P, jl, l - jl, Xd + static_cast<int64_t>(jl / kCB) * kCB * kCB, s_rl, inv_index(warp), lane);
    else
      chol_write_L_block(P, Lo, l, jl, (warp & 3) == 0 ? warp >> 2 : (warp == 11 ? 4 : warp - 8), 8, lane);
  }
}

// ---------------------------------------------------------------------------
// Q = Y L^-T for 64 rows of one problem per CTA, by 32-column panels:
//   T_J = Y_J - Q_<J L_J,<J^T        (4 rows x 2 columns per thread, K in float4 steps)
//   Q_J = T_J X_JJ^T,  X_JJ = L_JJ^-1 from chol3_kernel (1 row x 8 columns per thread)
// The 64 rows stay in shared memory; the rows of L that panel J+1 needs and
// X_J+1 are fetched with cp.async while panel J is computed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Stage rows c0 .. c0+w-1 of L (columns 0 .. c0) and X_J = L_JJ^-1.  One warp
// per row of L, lanes over float4 columns; 16-byte copies need l % 4 == 0
// (checked by the launcher).
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void trsm3_stage_L(const float* __restrict__ L, int l, int lqL, int J, float* Ls, int tid) {
  const int c0 = J * kCB, w = min(kCB, l - c0);
  const int warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  for (int c = warp; c < w; c += nw) {
    const float* src = L + static_cast<int64_t>(c0 + c) * l;
    for (int k4 = lane; k4 < c0 / 4; k4 += 32) cp_async16(Ls + c * lqL + 4 * k4, src + 4 * k4);
  }
}

__device__ __forceinline__ void trsm3_stage_X(const float* __restrict__ Xd, int J, float* Xs, int tid) {
  const float* xg = Xd + static_cast<int64_t>(J) * kCB * kCB;
  for (int e4 = tid; e4 < kCB * kCB / 4; e4 += blockDim.x) {
    const int i = e4 >> 3, c4 = e4 & 7;
    cp_async16(Xs + i * kLC + 4 * c4, xg + 4 * e4);
  }
}

constexpr int kR3 = 64;

__global__ void __launch_bounds__(256) trsm3_kernel(TrsmBatch tb, int l, int lqQ, int lqL,
                                                    const int* __restrict__ cond) {
  if (cond && *cond == 0) return;
  const TrsmProb& tp = tb.p[blockIdx.y];
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * kR3;
  if (r0 >= tp.rows) return;
  const int nrows = static_cast<int>(tp.rows - r0 < kR3 ? tp.rows - r0 : kR3);
  extern __shared__ float4 t3_smem4[];
  float* Qs = reinterpret_cast<float*>(t3_smem4);       // kR3 x lqQ
  float* Ls = Qs + kR3 * lqQ;                            // kCB x lqL
  float* Xb[2] = {Ls + kCB * lqL, Ls + kCB * lqL + kCB * kLC};
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float* __restrict__ Y = tp.Y;
  // rows of L beyond a partial last panel read as zero
  for (int e = tid; e < kCB * lqL; e += blockDim.x) Ls[e] = 0.f;
  {  // the 64 rows: every load of a thread issued before its stores
    const int q4 = lqQ / 4, nq = kR3 * q4;
    constexpr int kU = 8;
    for (int q0 = tid; q0 < nq; q0 += kU * 256) {
      float4 v[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int q = q0 + u * 256;
        const int r = q / q4, c4 = q - r * q4;
        v[u] = (q < nq && r < nrows && 4 * c4 < l) ? *reinterpret_cast<const float4*>(Y + (r0 + r) * l + 4 * c4)
                                                   : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int q = q0 + u * 256;
        if (q < nq) {
          const int r = q / q4, c4 = q - r * q4;
          *reinterpret_cast<float4*>(Qs + r * lqQ + 4 * c4) = v[u];
        }
      }
    }
  }
  const int np = (l + kCB - 1) / kCB;
  trsm3_stage_X(tp.Xd, 0, Xb[0], tid);
  cp_async_commit();
  const int ty = tid >> 4, tx = tid & 15;     // update: rows 4ty..4ty+3, columns tx, tx+16
  const int dr = tid >> 2, dg = tid & 3;      // diagonal: row dr, columns dg, dg+4, .., dg+28
  for (int J = 0; J < np; ++J) {
    const int c0 = J * kCB;
    float* Xs = Xb[J & 1];
    cp_async_wait_all();
    __syncthreads();
    if (c0 > 0) {
      float acc[4][2];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u][0] = acc[u][1] = 0.f;
      for (int k = 0; k < c0; k += 4) {
        float4 a4[4], b4[2];
#pragma unroll
        for (int u = 0; u < 4; ++u) a4[u] = *reinterpret_cast<const float4*>(Qs + (4 * ty + u) * lqQ + k);
#pragma unroll
        for (int v = 0; v < 2; ++v) b4[v] = *reinterpret_cast<const float4*>(Ls + (tx + 16 * v) * lqL + k);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 2; ++v) {
            acc[u][v] = fmaf(a4[u].x, b4[v].x, acc[u][v]);
            acc[u][v] = fmaf(a4[u].y, b4[v].y, acc[u][v]);
            acc[u][v] = fmaf(a4[u].z, b4[v].z, acc[u][v]);
            acc[u][v] = fmaf(a4[u].w, b4[v].w, acc[u][v]);
          }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v)
          if (c0 + tx + 16 * v < l) Qs[(4 * ty + u) * lqQ + c0 + tx + 16 * v] -= acc[u][v];
    }
    __syncthreads();
    // L rows and X for the next panel arrive while this panel's diagonal block is solved
    if (J + 1 < np) {
      trsm3_stage_L(tp.L, l, lqL, J + 1, Ls, tid);
      trsm3_stage_X(tp.Xd, J + 1, Xb[(J + 1) & 1], tid);
    }
    cp_async_commit();
    {
      float trow[kCB];
#pragma unroll
      for (int t4 = 0; t4 < kCB / 4; ++t4) {
        const float4 v4 = *reinterpret_cast<const float4*>(Qs + dr * lqQ + c0 + 4 * t4);
        trow[4 * t4] = v4.x;
        trow[4 * t4 + 1] = v4.y;
        trow[4 * t4 + 2] = v4.z;
        trow[4 * t4 + 3] = v4.w;
      }
      __syncthreads();
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) {
        const int c = 4 * cc + dg;   // the four dg of a warp read rows of X one stride apart: no bank conflict
        float v = 0.f;   // X_JJ is lower triangular (zero above the diagonal and beyond w)
#pragma unroll
        for (int t4 = 0; t4 < kCB / 4; ++t4) {
          const float4 x4 = *reinterpret_cast<const float4*>(Xs + c * kLC + 4 * t4);
          v = fmaf(trow[4 * t4], x4.x, v);
          v = fmaf(trow[4 * t4 + 1], x4.y, v);
          v = fmaf(trow[4 * t4 + 2], x4.z, v);
          v = fmaf(trow[4 * t4 + 3], x4.w, v);
        }
        if (c0 + c < l) Qs[dr * lqQ + c0 + c] = v;
      }
    }
  }
  __syncthreads();
  for (int r = warp; r < nrows; r += 8) {
    float4* dst = reinterpret_cast<float4*>(tp.Q + (r0 + r) * l);
    const float4* src = reinterpret_cast<const float4*>(Qs + r * lqQ);
    for (int c4 = lane; 4 * c4 < l; c4 += 32) dst[c4] = src[c4];
  }
}

// ---------------------------------------------------------------------------
// L^-1 from the Cholesky factor, one CTA (1024 threads) per 32-column
// block J.  Block row by block row (I = J, J+1, ..) the column block solves
//   L_II Li_IJ = -(sum_{K=J}^{I-1} L_IK Li_KJ)     (Li_JJ: L_JJ Li_JJ = I)
// by forward substitution in column order: warp c holds column c, lane i
// row i; for each t: x_t = b_t / L_tt (lane t), shuffled to the warp, then
// b_i -= L_it x_t for i > t.  The block sum is an FP32 dot product of L's
// rows with the column block (eight warps, four columns a thread), which is
// held transposed in shared memory (row c of Ct is column c of the block)
// so that both operands are read as float4; the diagonal block L_II is copied transposed so that the lanes
// read its columns without bank conflicts.  The rows of L below block J
// (columns j0 ..) are staged by cp.async, once when they fit, else block
// row by block row.  The result is written as TF32 high and low parts
// (Lh = the top 10 mantissa bits, Ll = Li - Lh, both l x l row-major, zero
// above the diagonal) for basis_tc_kernel.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16_li(float* dst, const float* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}

__global__ void __launch_bounds__(1024) linv_kernel(LinvBatch lb, int l, int whole, const int* __restrict__ cond) {
  if (cond && *cond == 0) return;
  const LinvProb& pb = lb.p[blockIdx.y];
  extern __shared__ float4 li_smem4[];
  const int J = blockIdx.x, j0 = J * kCB, nb = (l + kCB - 1) / kCB;
  const int cs = l - j0 + 4;                 // row stride of Ct and of the staged rows (a multiple of 4)
  float* Ct = reinterpret_cast<float*>(li_smem4);   // 32 x cs: Ct[c][r - j0] = Li(r, j0 + c)
  float* Dt = Ct + kCB * cs;                // 32 x 33: L_II transposed
  float* Ss = Dt + kCB * (kCB + 1);         // 32 x 33: the block sum, Ss[c][i]
  float* Pn = Ss + kCB * (kCB + 1);         // staged rows of L, columns j0 ..
  const int tid = threadIdx.x, c = tid >> 5, i = tid & 31;
  const float* __restrict__ L = pb.L;
  auto stage = [&](int r_first, int nrows, int ncols4) {
    for (int q = tid; q < nrows * ncols4; q += 1024) {
      const int r = q / ncols4, c4 = q - r * ncols4;
      cp_async16_li(Pn + r * cs + 4 * c4, L + static_cast<int64_t>(r_first + r) * l + j0 + 4 * c4);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  };
  if (whole) stage(j0, l - j0, (l - j0) / 4);   // rows j0 .. l-1
  for (int I = J; I < nb; ++I) {
    const int i0 = I * kCB, wI = min(kCB, l - i0), kw = i0 - j0;   // kw: a multiple of 32
    if (!whole) stage(i0, wI, (kw + wI + 3) / 4);                  // rows of block I, columns j0 .. i0 + wI
    __syncthreads();
    const float* prow = Pn + (whole ? kw + i : i) * cs;   // row i0 + i of L (columns j0 ..)
    // the diagonal block, transposed: Dt[t][i] = L(i0 + i, i0 + t)
    Dt[c * (kCB + 1) + i] = (i < wI && c < wI) ? prow[kw + c] : 0.f;
    if (I > J && tid < 256) {
      // the block sum, by the first eight warps: thread (row ii, columns
      // 4 cg .. +3), each row of L read once for four columns
      const int ii = tid & 31, cg = tid >> 5;
      float a[4] = {0.f, 0.f, 0.f, 0.f};
      if (ii < wI) {
        const float* pr = Pn + (whole ? kw + ii : ii) * cs;
#pragma unroll 2
        for (int k = 0; k < kw; k += 4) {
          const float4 lv = *reinterpret_cast<const float4*>(pr + k);
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const float4 cv = *reinterpret_cast<const float4*>(Ct + (4 * cg + v) * cs + k);
            a[v] = fmaf(lv.x, cv.x, a[v]);
            a[v] = fmaf(lv.y, cv.y, a[v]);
            a[v] = fmaf(lv.z, cv.z, a[v]);
            a[v] = fmaf(lv.w, cv.w, a[v]);
          }
        }
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) Ss[(4 * cg + v) * (kCB + 1) + ii] = a[v];
    }
    const float rv = i < wI ? 1.0f / prow[kw + i] : 1.0f;   // 1 / L_ii
    __syncthreads();   // Dt and Ss complete
    float b = I == J ? (i == c ? 1.f : 0.f) : -Ss[c * (kCB + 1) + i];
#pragma unroll 4
    for (int t = 0; t < wI; ++t) {
      const float xt = __shfl_sync(0xffffffffu, b * rv, t);
      if (i > t && i < wI) b = fmaf(-Dt[t * (kCB + 1) + i], xt, b);
    }
    if (i < wI) Ct[c * cs + kw + i] = b * rv;
    __syncthreads();
  }
  // column block J of Lh, Ll: rows 0 .. l-1, zeros above row j0; thread:
  // row tid / 8 (+ 128 n), columns 4 (tid mod 8) .. +3
  const int jq = 4 * (tid & 7), col = j0 + jq;
  if (col < l) {
    for (int r = tid >> 3; r < l; r += 128) {
      float h[4], o[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float v = r >= j0 ? Ct[(jq + u) * cs + r - j0] : 0.f;
        h[u] = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
        o[u] = v - h[u];
      }
      *reinterpret_cast<float4*>(pb.Lh + static_cast<int64_t>(r) * l + col) = make_float4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<float4*>(pb.Ll + static_cast<int64_t>(r) * l + col) = make_float4(o[0], o[1], o[2], o[3]);
    }
  }
}

}  // namespace

size_t gram_part_floats(int l) {
  // splits * tiles <= ~2 * 152 per problem, two problems
  (void)l;
  return static_cast<size_t>(2) * 320 * kGT * kGT;
}

lramm_status launch_gram(GramBatch gb, int l, float* part, cudaStream_t s, const int* cond) {
  const int nt = (l + kGT - 1) / kGT;
  const int ntiles = nt * (nt + 1) / 2;
  int64_t rows = 0;
  for (int i = 0; i < gb.n; ++i) rows = gb.p[i].rows > rows ? gb.p[i].rows : rows;
  bool vec = l % 4 == 0;
  for (int i = 0; i < gb.n; ++i) vec = vec && (reinterpret_cast<uintptr_t>(gb.p[i].Y) & 15) == 0;
  // 64-thread CTAs (8 x 8 per thread) run several per SM: aim at ~6 per SM
  const int want = vec ? 6 * num_sms() : 2 * num_sms();
  int splits = static_cast<int>((want / gb.n + ntiles - 1) / ntiles);
  if (splits > 320 / ntiles) splits = 320 / ntiles;
  if (splits < 1) splits = 1;
  int64_t rps = ceil_div(ceil_div(rows, splits), 16) * 16;
  if (rps < 64) rps = 64;
  splits = static_cast<int>(ceil_div(rows, rps));
  if (static_cast<size_t>(gb.n) * splits * ntiles > 2 * 320) return LRAMM_ERR_UNSUPPORTED;
  if (vec)
    gram_partial8_kernel<<<dim3(ntiles, splits, gb.n), 64, 0, s>>>(gb, l, ntiles, splits, rps, part, cond);
  else
    gram_partial_kernel<false><<<dim3(ntiles, splits, gb.n), 256, 0, s>>>(gb, l, ntiles, splits, rps, part, cond);
  LRAMM_TRY(last_launch());
  const int64_t g = ceil_div(static_cast<int64_t>(ntiles) * kGT * kGT / 4 * gb.n, 64);
  gram_reduce_kernel<<<static_cast<unsigned>(g), 64, 0, s>>>(gb, l, ntiles, splits, part, cond);
  return last_launch();
}

static const int kSmemMaxO = 232448 - 1024;

lramm_status launch_chol2(SmallBatch bt, int l, float shift_rel, int* status, cudaStream_t s) {
  const size_t smem = sizeof(float) * static_cast<size_t>(l) * (l + 1) / 2;
  if (smem > static_cast<size_t>(kSmemMaxO)) return LRAMM_ERR_UNSUPPORTED;
  LRAMM_CUDA_TRY(smem_cap(chol2_kernel, static_cast<int>(smem)));
  chol2_kernel<<<bt.n, 1024, smem, s>>>(bt, l, shift_rel, status);
  return last_launch();
}

lramm_status launch_trsm_panel(SmallBatch bt, int l, cudaStream_t s) {
  const int lq = static_cast<int>(round_up(l, kTP)) + 1;
  const size_t smem = sizeof(float) * (static_cast<size_t>(kTR) * lq + static_cast<size_t>(kTP) * (lq + 4) +
                                       static_cast<size_t>(kTP) * (kTP + 1));
  if (smem > static_cast<size_t>(kSmemMaxO)) return LRAMM_ERR_UNSUPPORTED;
  LRAMM_CUDA_TRY(
      smem_cap(trsm_panel_kernel, static_cast<int>(smem)));
  int64_t rows = 0;
  for (int i = 0; i < bt.n; ++i) rows = bt.p[i].rows > rows ? bt.p[i].rows : rows;
  trsm_panel_kernel<<<dim3(static_cast<unsigned>(ceil_div(rows, kTR)), bt.n), 256, smem, s>>>(bt, l, lq);
  return last_launch();
}

size_t chol3_smem(int l) {
  const size_t np = static_cast<size_t>(l) * (l + 1) / 2;
  const size_t lp = round_up(l, 4) + 4;
  return sizeof(float) * (round_up(np, 4) + kCB * lp + kCB * kLC);
}

// The tensor-core variant: no transposed panel, two 32 KB swizzled panel
// copies at a 1024-byte boundary.
size_t chol3_tc_smem(int l) {
  const size_t np = static_cast<size_t>(l) * (l + 1) / 2;
  return sizeof(float) * (round_up(np, 4) + kCB * kLC) + 1024 + 2 * 256 * 128;
}

bool chol3_supported(int l) { return l >= 4 && l % 4 == 0 && l - kCB <= 256 && chol3_smem(l) <= static_cast<size_t>(kSmemMaxO); }

lramm_status launch_chol3(CholBatch cb, int l, float shift_rel, int* status, cudaStream_t s, const int* cond,
                          float shift_big_rel) {
  if (!chol3_supported(l)) return LRAMM_ERR_UNSUPPORTED;
  if (chol3_tc_smem(l) <= static_cast<size_t>(kSmemMaxO)) {
    const size_t smem = chol3_tc_smem(l);
    LRAMM_CUDA_TRY(smem_cap(chol3_kernel<true>, static_cast<int>(smem)));
    // Without the diagonal-block inversions (eight warps of their own) 384
    // threads do the rest: three quarters of the SM's registers, so that the
    // CTA finds room beside a concurrent range-finder product's CTA on its SM
    // instead of waiting for an empty SM.  The panel solve takes one thread
    // per row below the diagonal block (at most 256: l - 32 <= 256).
    bool inv = false;
    for (int i = 0; i < cb.n; ++i) inv = inv || cb.p[i].Xd != nullptr;
    chol3_kernel<true><<<cb.n, inv ? 512 : 384, smem, s>>>(cb, l, shift_rel, shift_big_rel, status, cond);
    return last_launch();
  }
  const size_t smem = chol3_smem(l);
  LRAMM_CUDA_TRY(smem_cap(chol3_kernel<false>, static_cast<int>(smem)));
  chol3_kernel<false><<<cb.n, 512, smem, s>>>(cb, l, shift_rel, shift_big_rel, status, cond);
  return last_launch();
}

lramm_status launch_trsm3(TrsmBatch tb, int l, cudaStream_t s, const int* cond) {
  // float4 staging: rows of Y, Q and L start on 16-byte boundaries
  if (l % 4 != 0) return LRAMM_ERR_UNSUPPORTED;
  for (int i = 0; i < tb.n; ++i)
    if ((reinterpret_cast<uintptr_t>(tb.p[i].Y) | reinterpret_cast<uintptr_t>(tb.p[i].Q) |
         reinterpret_cast<uintptr_t>(tb.p[i].L) | reinterpret_cast<uintptr_t>(tb.p[i].Xd)) & 15)
      return LRAMM_ERR_UNSUPPORTED;
  const int lqQ = static_cast<int>(round_up(l, kCB)) + 4;   // panel writes reach round_up(l, 32)
  const int lqL = static_cast<int>(round_up(l > kCB ? l - kCB : 4, kCB)) + 4;
  const size_t smem = sizeof(float) * (static_cast<size_t>(kR3) * lqQ + static_cast<size_t>(kCB) * lqL + 2 * kCB * kLC);
  if (smem > static_cast<size_t>(kSmemMaxO)) return LRAMM_ERR_UNSUPPORTED;
  LRAMM_CUDA_TRY(smem_cap(trsm3_kernel, static_cast<int>(smem)));
  int64_t rows = 0;
  for (int i = 0; i < tb.n; ++i) rows = tb.p[i].rows > rows ? tb.p[i].rows : rows;
  trsm3_kernel<<<dim3(static_cast<unsigned>(ceil_div(rows, kR3)), tb.n), 256, smem, s>>>(tb, l, lqQ, lqL, cond);
  return last_launch();
}

lramm_status launch_linv(LinvBatch lb, int l, cudaStream_t s, const int* cond) {
  if (l % 4 != 0 || l < 4) return LRAMM_ERR_UNSUPPORTED;
  for (int i = 0; i < lb.n; ++i)
    if ((reinterpret_cast<uintptr_t>(lb.p[i].L) | reinterpret_cast<uintptr_t>(lb.p[i].Lh) |
         reinterpret_cast<uintptr_t>(lb.p[i].Ll)) & 15)
      return LRAMM_ERR_UNSUPPORTED;
  // the transposed column block and the rows of L below block 0 (the
  // largest): all at once when they fit, else one block row at a time
  const size_t nbk = ceil_div(l, kCB);
  const size_t whole_smem = sizeof(float) * ((static_cast<size_t>(kCB) + l) * (l + 4) + 2 * kCB * (kCB + 1));
  const size_t step_smem = sizeof(float) * (2 * static_cast<size_t>(kCB) * (l + 4) + 2 * kCB * (kCB + 1));
  const int whole = whole_smem <= static_cast<size_t>(kSmemMaxO) ? 1 : 0;
  const size_t smem = whole ? whole_smem : step_smem;
  if (smem > static_cast<size_t>(kSmemMaxO)) return LRAMM_ERR_UNSUPPORTED;
  LRAMM_CUDA_TRY(smem_cap(linv_kernel, static_cast<int>(smem)));
  linv_kernel<<<dim3(static_cast<unsigned>(nbk), lb.n), 1024, smem, s>>>(lb, l, whole, cond);
  return last_launch();
}


// ---------------------------------------------------------------------------
// Cholesky of Grams too large for one CTA's shared memory (chol3_kernel
// stops at l = 288), two-level with h = min(288, round_up(l/2, 32)):
//   G + shift I = [G11 G21^T; G21 G22],  L11 = chol(G11),  L21 = G21 L11^-T,
//   L22 = chol(G22 - L21 L21^T),  L = [L11 0; L21 L22].
// The shift comes from the whole matrix's diagonal before the split.  h is a
// multiple of 32, so the inverted 32 x 32 diagonal blocks of L11 and L22 are
// those of L, in order, and the panel solve of the tall sketch runs on L
// unchanged.  Scratch per problem (2 l^2 floats):
//   G11 h x h | G21 m x h | S m x m | L11 h x h | L21 m x h | L22 m x m, m = l - h.
// ---------------------------------------------------------------------------
int chol_split_h(int l) { return chol_split_h_dev(l); }

bool chol_split_supported(int l) {
  if (l % 4 != 0 || l <= 288) return false;
  const int h = chol_split_h(l), m = l - h;
  return m >= 4 && chol3_supported(h) && chol3_supported(m);
}

size_t chol_split_scratch_floats(int l) { return 2 * static_cast<size_t>(l) * l; }

struct SplitPtrs {
  float *G11, *G21, *S, *L11, *L21, *L22;
};

__host__ __device__ inline SplitPtrs split_ptrs(float* w, int l) {
  const int64_t h = chol_split_h_dev(l), m = l - h;
  SplitPtrs p;
  p.G11 = w;
  p.G21 = p.G11 + h * h;
  p.S = p.G21 + m * h;
  p.L11 = p.S + m * m;
  p.L21 = p.L11 + h * h;
  p.L22 = p.L21 + m * h;
  return p;
}

__global__ void __launch_bounds__(256) chol_split_prep_kernel(CholBatch cb, SplitScratch sc, int l, float shift_rel,
                                                              const int* __restrict__ cond) {
  if (cond && *cond == 0) return;
  const CholProb& cp = cb.p[blockIdx.y];
  const float* __restrict__ G = cp.G;
  __shared__ float s_red[8];
  float md = 0.f;
  for (int i = threadIdx.x; i < l; i += blockDim.x) md = fmaxf(md, G[static_cast<int64_t>(i) * l + i]);
  md = warp_max_o(md);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = md;
  __syncthreads();
  float mx = 0.f;
#pragma unroll
  for (int w = 0; w < 8; ++w) mx = fmaxf(mx, s_red[w]);
  const float shift = shift_rel * mx;
  const int h = chol_split_h_dev(l), m = l - h;
  const SplitPtrs sp = split_ptrs(sc.w[blockIdx.y], l);
  const int64_t n = static_cast<int64_t>(l) * l;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(e / l), j = static_cast<int>(e - static_cast<int64_t>(i) * l);
    const float v = G[e] + (i == j ? shift : 0.f);
    if (i < h) {
      if (j < h) sp.G11[i * h + j] = v;
    } else if (j < h) {
      sp.G21[(i - h) * h + j] = v;
    } else {
      sp.S[(i - h) * m + (j - h)] = v;
    }
  }
}

__global__ void __launch_bounds__(256) chol_split_assemble_kernel(CholBatch cb, SplitScratch sc, int l,
                                                                  const int* __restrict__ cond) {
  if (cond && *cond == 0) return;
  float* __restrict__ Lo = cb.p[blockIdx.y].L;
  const int h = chol_split_h_dev(l), m = l - h;
  const SplitPtrs sp = split_ptrs(sc.w[blockIdx.y], l);
  const int64_t n = static_cast<int64_t>(l) * l;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(e / l), j = static_cast<int>(e - static_cast<int64_t>(i) * l);
    float v;
    if (i < h) v = j < h ? sp.L11[i * h + j] : 0.f;
    else v = j < h ? sp.L21[(i - h) * h + j] : sp.L22[(i - h) * m + (j - h)];
    Lo[e] = v;
  }
}

lramm_status launch_chol_split(CholBatch cb, SplitScratch sc, int l, float shift_rel, int* status, cudaStream_t s,
                               const int* cond) {
  if (!chol_split_supported(l)) return LRAMM_ERR_UNSUPPORTED;
  const int h = chol_split_h(l), m = l - h;
  const dim3 grid(static_cast<unsigned>(ceil_div(static_cast<int64_t>(l) * l, 256 * 8)), cb.n);
  chol_split_prep_kernel<<<grid, 256, 0, s>>>(cb, sc, l, shift_rel, cond);
  LRAMM_TRY(last_launch());
  CholBatch c1{}, c2{};
  TrsmBatch t1{};
  c1.n = c2.n = t1.n = cb.n;
  for (int i = 0; i < cb.n; ++i) {
    const SplitPtrs sp = split_ptrs(sc.w[i], l);
    c1.p[i] = CholProb{sp.G11, sp.L11, cb.p[i].Xd, cb.p[i].brk, cb.p[i].brk_any, cb.p[i].brk_count};
    t1.p[i] = TrsmProb{sp.G21, sp.L21, sp.L11, cb.p[i].Xd, m};
    c2.p[i] = CholProb{sp.S, sp.L22, cb.p[i].Xd + static_cast<int64_t>(h / kCB) * kCB * kCB, cb.p[i].brk,
                       cb.p[i].brk_any, cb.p[i].brk_count};
  }
  LRAMM_TRY(launch_chol3(c1, h, 0.f, status, s, cond));
  LRAMM_TRY(launch_trsm3(t1, h, s, cond));
  for (int i = 0; i < cb.n; ++i) {
    const SplitPtrs sp = split_ptrs(sc.w[i], l);
    LRAMM_TRY(sgemm(0, 1, m, m, h, -1.f, sp.L21, h, 0, sp.L21, h, 1.f, sp.S, m, s, cond));   // S = G22 - L21 L21^T
  }
  LRAMM_TRY(launch_chol3(c2, m, 0.f, status, s, cond));
  chol_split_assemble_kernel<<<grid, 256, 0, s>>>(cb, sc, l, cond);
  return last_launch();
}

__global__ void copy_cond_kernel(const float* __restrict__ src, float* __restrict__ dst, int64_t n,
                                 const int* __restrict__ cond) {
  if (*cond == 0) return;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    dst[e] = src[e];
}

lramm_status launch_copy_cond(const float* src, float* dst, int64_t n, const int* cond, cudaStream_t s) {
  if (n <= 0) return LRAMM_OK;
  int64_t g = ceil_div(n, 256);
  if (g > num_sms() * 4) g = num_sms() * 4;
  copy_cond_kernel<<<static_cast<unsigned>(g), 256, 0, s>>>(src, dst, n, cond);
  return last_launch();
}

}  // namespace lramm
