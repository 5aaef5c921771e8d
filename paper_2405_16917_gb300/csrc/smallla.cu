// Small dense linear algebra of the randomized SVD (sizes l x l, l = r + p):
//   * Cholesky of the Gram matrix for CholeskyQR (orthonormalisation of the
//     sketch, Sec. 2.2: "a matrix Q with r orthonormal columns"),
//   * the triangular solve Q = Y L^-T that applies it to the tall sketch,
//   * one-sided Jacobi SVD of the l x l triangular factor (the SVD of
//     B = Q^* A in Algorithm 1, taken on the R factor of B^T = P R),
//   * sorting / truncation of the SVD to rank r.
// All FP32.  Every loop has a fixed trip count; nothing waits on a flag.
#include <float.h>

#include <cooperative_groups.h>

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
__global__ void __launch_bounds__(1024) chol_kernel(SmallBatch bt, int l, float shift_rel, int* status) {
  const float* __restrict__ G = bt.p[blockIdx.x].in;
  float* __restrict__ L = bt.p[blockIdx.x].out;
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
__global__ void __launch_bounds__(1024) trsm_rows_kernel(SmallBatch bt, int l) {
  const float* __restrict__ Y = bt.p[blockIdx.y].in;
  float* __restrict__ Q = bt.p[blockIdx.y].out;
  const float* __restrict__ L = bt.p[blockIdx.y].aux;
  const int64_t rows = bt.p[blockIdx.y].rows;
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

// Sort columns by descending norm (sigma) and write the rank-r outputs.
// blockIdx.y = problem; blockIdx.x = a slice of 32 output rows.  Every CTA
// recomputes the l norms and the ranking (l^2 work, cheap) so that the
// row-major S1 / S2 rows can be written coalesced (consecutive threads,
// consecutive output columns p).  Ties are broken by column index.
constexpr int kFinRows = 32;
constexpr int kFinMaxL = 576;   // largest l of the SVD form (multiple of 32)

__global__ void __launch_bounds__(256) svd_finalize_kernel(FinalBatch fb, int l, int r) {
  const FinalProb& fp = fb.p[blockIdx.y];
  const float* __restrict__ M = fp.M;
  const float* __restrict__ V = fp.V;
  extern __shared__ float sm[];
  float* nrm = sm;                                  // l
  int* pos = reinterpret_cast<int*>(sm + l);        // l
  int* inv = pos + l;                               // r: column holding rank p
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  // column norms, four columns per warp at a time with every load of the
  // four issued before the sums (l <= kFinMaxL): the same per-column
  // summation order as one column at a time
  for (int j0 = warp; j0 < l; j0 += 4 * nw) {
    float v[4][kFinMaxL / 32];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + c * nw;
#pragma unroll
      for (int u = 0; u < kFinMaxL / 32; ++u) {
        const int i = lane + 32 * u;
        v[c][u] = (j < l && i < l) ? M[(int64_t)j * l + i] : 0.f;
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + c * nw;
      float s = 0.f;
#pragma unroll
      for (int u = 0; u < kFinMaxL / 32; ++u)
        if (lane + 32 * u < l) s = fmaf(v[c][u], v[c][u], s);
      s = warp_sum(s);
      if (lane == 0 && j < l) nrm[j] = sqrtf(s);
    }
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
    if (rank < r) inv[rank] = j;
  }
  __syncthreads();
  if (blockIdx.x == 0)
    for (int p = tid; p < r; p += blockDim.x) fp.sig[p] = nrm[inv[p]];
  const int i0 = blockIdx.x * kFinRows, i1 = min(l, i0 + kFinRows);
  const int ne = (i1 - i0) * r;
  // four outputs per thread per step, their loads issued together
  for (int e0 = tid; e0 < ne; e0 += 4 * blockDim.x) {
    float mv[4], vv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + u * blockDim.x;
      const int i = i0 + e / r, p = e - (e / r) * r;
      const int j = e < ne ? inv[p] : 0;
      mv[u] = e < ne ? M[(int64_t)j * l + i] : 0.f;
      vv[u] = e < ne ? V[(int64_t)j * l + i] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e >= ne) break;
      const int i = i0 + e / r, p = e - (e / r) * r;
      const float sj = nrm[inv[p]];
      const float u_scale = fp.s1_sigma ? 1.0f : (sj > 0.f ? 1.0f / sj : 0.f);
      const float v_scale = fp.s2_sigma ? sj : 1.0f;
      const float o1 = mv[u] * u_scale, o2 = vv[u] * v_scale;
      fp.S1[(int64_t)i * r + p] = o1;
      fp.S2[(int64_t)i * r + p] = o2;
      fp.S1T[(int64_t)p * l + i] = o1;
      fp.S2T[(int64_t)p * l + i] = o2;
    }
  }
}

// ---------------------------------------------------------------------------
// One-sided Jacobi on a thread-block cluster, columns resident in shared
// memory.  The l columns (padded with zero columns to 2*C*b) form 2C blocks
// of b columns; CTA c of the cluster holds two of them (a "top" and a
// "bottom" slot) in three b-column buffers (two in use, one free).  A sweep
// is 2C-1 block rounds; in each, a CTA rotates every (top, bottom) column
// pair -- b rounds of b disjoint pairs, one warp per pair, CTA barriers only
// -- and in the first block round also every pair inside its two blocks.
// Between block rounds the blocks circulate through distributed shared
// memory in round-robin (circle) order: the top of CTA 0 stays, every other
// block moves one place along the ring B0 -> T1 -> T2 ... -> T(C-1) ->
// B(C-1) -> ... -> B0, so in 2C-1 block rounds every pair of blocks meets
// once.  A pair (a, b) is rotated when |a.b| > tol |a| |b|; the sweep loop
// stops after a sweep without rotations anywhere in the cluster, or after
// max_sweeps (then LRAMM_WARN_NOCONV is latched).  All loops have fixed
// bounds and every CTA of a cluster takes the same branches.
// ---------------------------------------------------------------------------
namespace cg = cooperative_groups;

// Physical buffers (top, bottom, free) of cluster rank `rank` after e moves.
__device__ __forceinline__ void jc_bufs(int rank, int e, int& t, int& bo, int& f) {
  if (rank == 0) {
    t = 0; bo = 1; f = 2;
    return;
  }
  const int m = e % 3;
  if (m == 0) { t = 0; bo = 1; f = 2; }
  else if (m == 1) { t = 2; bo = 0; f = 1; }
  else { t = 1; bo = 2; f = 0; }
}

// Rotate columns (a, b) (M part at the pointer, V part ls floats further)
// so that their inner product vanishes; one warp.  Returns whether it did;
// rmax takes the largest relative inner product |a.b| / (|a| |b|) met.
__device__ __forceinline__ bool jc_rotate(float* __restrict__ a, float* __restrict__ b, int l, int ls,
                                          float tol, int lane, float& rmax) {
  float al = 0.f, be = 0.f, ga = 0.f;
  for (int i = lane; i < l; i += 32) {
    const float x = a[i], y = b[i];
    al = fmaf(x, x, al);
    be = fmaf(y, y, be);
    ga = fmaf(x, y, ga);
  }
  al = warp_sum(al);
  be = warp_sum(be);
  ga = warp_sum(ga);
  const float nab = sqrtf(al) * sqrtf(be);
  if (nab > 0.f && fabsf(ga) / nab > rmax) rmax = fabsf(ga) / nab;
  if (!(fabsf(ga) > tol * nab)) return false;
  const float zeta = (be - al) / (2.0f * ga);
  const float tt = fabsf(zeta) > 1e18f ? 0.5f / zeta
                                       : copysignf(1.0f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.0f)));
  const float c = 1.0f / sqrtf(fmaf(tt, tt, 1.0f));
  const float s = c * tt;
  // x' = c x - s y, y' = s x + c y applied as x - s (y + tau x) and
  // y + s (x - tau y), tau = s / (1 + c): for small angles fl(c) = 1 and the
  // plain form would dilate both columns by 1 + t^2.
  const float tau = s / (1.0f + c);
  for (int i = lane; i < l; i += 32) {
    const float x = a[i], y = b[i];
    a[i] = x - s * fmaf(tau, x, y);
    b[i] = y + s * fmaf(-tau, y, x);
  }
  float* va = a + ls;
  float* vb = b + ls;
  for (int i = lane; i < l; i += 32) {
    const float x = va[i], y = vb[i];
    va[i] = x - s * fmaf(tau, x, y);
    vb[i] = y + s * fmaf(-tau, y, x);
  }
  return true;
}

__global__ void __launch_bounds__(1024)
jacobi_cluster_kernel(JacobiBatch jb, int l, int ls, int b, int max_sweeps, float tol, int* status) {
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int prob = blockIdx.x / C;
  float* __restrict__ Mg = jb.M[prob];
  float* __restrict__ Vg = jb.V[prob];
  extern __shared__ float4 jc_smem4[];
  float* sm = reinterpret_cast<float*>(jc_smem4);
  const int64_t bufsz = (int64_t)b * 2 * ls;  // floats per buffer
  __shared__ int s_flags[16];
  __shared__ int s_ids[32];
  __shared__ int s_rot;
  __shared__ int s_rmax;   // bits of the sweep's largest relative inner product (non-negative)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int nslots = 2 * C;

  if (tid < nslots) s_ids[tid] = tid;
  // initial blocks: top = block 2 rank (buffer 0), bottom = block 2 rank + 1 (buffer 1)
  for (int half = 0; half < 2; ++half) {
    float* buf = sm + half * bufsz;
    const int blk = 2 * rank + half;
    for (int j = warp; j < b; j += nw) {
      const int g = blk * b + j;
      float* col = buf + (int64_t)j * 2 * ls;
      for (int i = lane; i < ls; i += 32) {
        col[i] = (g < l && i < l) ? Mg[(int64_t)g * l + i] : 0.f;
        col[ls + i] = (g < l && i == g) ? 1.f : 0.f;
      }
    }
  }
  cluster.sync();

  int e = 0;  // block moves so far
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) {
      s_rot = 0;
      s_rmax = 0;
    }
    float rmax = 0.f;
    __syncthreads();
    for (int br = 0; br < 2 * C - 1; ++br) {
      int bt_, bb_, bf_;
      jc_bufs(rank, e, bt_, bb_, bf_);
      float* topb = sm + bt_ * bufsz;
      float* botb = sm + bb_ * bufsz;
      if (br == 0) {  // pairs inside each of the two blocks (circle method on b columns)
        const int be = b + (b & 1), half = be / 2;
        for (int t = 0; t < be - 1; ++t) {
          for (int kp = warp; kp < 2 * half; kp += nw) {
            float* base = kp < half ? topb : botb;
            const int k = kp % half;
            int x, y;
            if (k == 0) {
              x = 0;
              y = 1 + t % (be - 1);
            } else {
              x = 1 + (t + k) % (be - 1);
              y = 1 + (t - k + (be - 1)) % (be - 1);
            }
            if (x >= b || y >= b) continue;
            if (jc_rotate(base + (int64_t)x * 2 * ls, base + (int64_t)y * 2 * ls, l, ls, tol, lane, rmax) &&
                lane == 0)
              s_rot = 1;
          }
          __syncthreads();
        }
      }
      for (int j = 0; j < b; ++j) {  // top column i against bottom column (i + j) mod b
        for (int i = warp; i < b; i += nw) {
          const int k = (i + j) % b;
          if (jc_rotate(topb + (int64_t)i * 2 * ls, botb + (int64_t)k * 2 * ls, l, ls, tol, lane, rmax) &&
              lane == 0)
            s_rot = 1;
        }
        __syncthreads();
      }
      if (C > 1) {
        cluster.sync();  // every CTA has finished rotating the blocks it is about to hand on
        // move 1: every CTA but 0 pulls its new top into its free buffer
        if (rank >= 1) {
          int st, sb, sf;
          jc_bufs(rank - 1, e, st, sb, sf);
          const float4* src =
              cluster.map_shared_rank(reinterpret_cast<float4*>(sm + (rank == 1 ? sb : st) * bufsz), rank - 1);
          float4* dst = reinterpret_cast<float4*>(sm + bf_ * bufsz);
          for (int64_t q = tid; q < bufsz / 4; q += blockDim.x) dst[q] = src[q];
        }
        cluster.sync();
        // move 2: every CTA but the last pulls its new bottom from the next CTA
        // (the last one's new bottom is its old top, already in place)
        if (rank <= C - 2) {
          int st, sb, sf;
          jc_bufs(rank + 1, e, st, sb, sf);
          const float4* src = cluster.map_shared_rank(reinterpret_cast<float4*>(sm + sb * bufsz), rank + 1);
          float4* dst = reinterpret_cast<float4*>(sm + (rank == 0 ? bb_ : bt_) * bufsz);
          for (int64_t q = tid; q < bufsz / 4; q += blockDim.x) dst[q] = src[q];
        }
        if (tid == 0) {  // slot -> block bookkeeping, identical on every CTA
          int nid[32];
          nid[0] = s_ids[0];
          nid[2] = s_ids[1];
          for (int c = 2; c < C; ++c) nid[2 * c] = s_ids[2 * c - 2];
          nid[2 * C - 1] = s_ids[2 * C - 2];
          for (int c = 0; c <= C - 2; ++c) nid[2 * c + 1] = s_ids[2 * c + 3];
          for (int q = 0; q < nslots; ++q) s_ids[q] = nid[q];
        }
        cluster.sync();
        ++e;
      }
    }
    // did any CTA of the cluster rotate in this sweep, and how far from
    // orthogonal was the worst pair?  Stop after a sweep without rotations
    // or one whose largest relative inner product is below stopq tol (the
    // next sweep would leave inner products of the order of its square).
    if (lane == 0) atomicMax(&s_rmax, __float_as_int(rmax));
    __syncthreads();
    if (tid < C) *cluster.map_shared_rank(&s_flags[rank], tid) = s_rot ? s_rmax : -1;
    cluster.sync();
    int any = 0, mx = 0;
    for (int c = 0; c < C; ++c) {
      any |= s_flags[c] >= 0;
      mx = max(mx, s_flags[c]);
    }
    cluster.sync();
    if (!any || !(__int_as_float(mx) > jb.stopq * tol)) break;
  }
  if (sweep >= max_sweeps && tid == 0 && rank == 0) set_status(status, LRAMM_WARN_NOCONV);
  if (tid == 0 && rank == 0 && status) status[1 + jb.info0 + prob] = sweep < max_sweeps ? sweep + 1 : sweep;  // diagnostics
  int bt_, bb_, bf_;
  jc_bufs(rank, e, bt_, bb_, bf_);
  for (int half = 0; half < 2; ++half) {
    const float* buf = sm + (half == 0 ? bt_ : bb_) * bufsz;
    const int blk = s_ids[2 * rank + half];
    for (int j = warp; j < b; j += nw) {
      const int g = blk * b + j;
      if (g >= l) continue;
      const float* col = buf + (int64_t)j * 2 * ls;
      for (int i = lane; i < l; i += 32) {
        Mg[(int64_t)g * l + i] = col[i];
        Vg[(int64_t)g * l + i] = col[ls + i];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// The same one-sided Jacobi schedule on a cluster of up to 16 CTAs with two
// warps per column pair: C = min(16, ceil(l/16)) CTAs, blocks of b <= 10
// columns, 64 b threads per CTA.  Thread p of pair group g owns rows
// p, p + 64, ... (RP of them) of both columns of its pair; the three inner
// products are reduced by warp shuffles and summed over the group's two
// warps through shared memory behind a 64-thread named barrier (the same
// order in every thread, so the whole group takes identical decisions).
// During a block round group g keeps top column g in registers and meets
// bottom column (g + j) mod b in round j.  Rotation formulas, threshold,
// round-robin order and stopping rule are those of jacobi_cluster_kernel.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void group_bar(int id) {
  asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory");
}

// Stopping rule of the cluster Jacobi: a sweep whose largest relative inner
// product stays below jb.stopq * tol is the last one (callers pass
// kJacobiQuad = 20 for a converged SVD).

template <int RP, int GW, bool WV = true>
__device__ __forceinline__ bool jc2_rotate(float (&xm)[RP], float (&xv)[RP], float (&ym)[RP], float (&yv)[RP],
                                           float tol, int grp, int wig, int lane, float (*s_part)[2][4],
                                           float& rmax) {
  float al = 0.f, be = 0.f, ga = 0.f;
#pragma unroll
  for (int u = 0; u < RP; ++u) {
    al = fmaf(xm[u], xm[u], al);
    be = fmaf(ym[u], ym[u], be);
    ga = fmaf(xm[u], ym[u], ga);
  }
  // Three warp sums with six shuffles: the halves of the warp trade (al, be)
  // and then (that, ga) so that each lane carries one quantity; the totals
  // end in lanes 0 (al), 8 (ga) and 16 (be).
  {
    const bool hi16 = lane & 16, hi8 = lane & 8;
    float v = hi16 ? be : al;
    const float u = hi16 ? al : be;
    v += __shfl_xor_sync(0xffffffffu, u, 16);
    ga += __shfl_xor_sync(0xffffffffu, ga, 16);
    float x = hi8 ? ga : v;
    const float y = hi8 ? v : ga;
    x += __shfl_xor_sync(0xffffffffu, y, 8);
    x += __shfl_xor_sync(0xffffffffu, x, 4);
    x += __shfl_xor_sync(0xffffffffu, x, 2);
    x += __shfl_xor_sync(0xffffffffu, x, 1);
    if (GW == 1) {  // one warp per pair: broadcast the three totals
      al = __shfl_sync(0xffffffffu, x, 0);
      be = __shfl_sync(0xffffffffu, x, 16);
      ga = __shfl_sync(0xffffffffu, x, 8);
    } else {
      if (lane == 0) s_part[grp][wig][0] = x;
      if (lane == 16) s_part[grp][wig][1] = x;
      if (lane == 8) s_part[grp][wig][2] = x;
    }
  }
  if (GW == 2) {  // two warps per pair: add the warps' totals (same order everywhere)
    group_bar(1 + grp);
    al = s_part[grp][0][0] + s_part[grp][1][0];
    be = s_part[grp][0][1] + s_part[grp][1][1];
    ga = s_part[grp][0][2] + s_part[grp][1][2];
  }
  // Threshold and angle in fast arithmetic: the angle only has to be close
  // (an inexact one leaves a small inner product for the next sweep); the
  // rotation stays orthogonal to working precision because s and c come
  // from the same t and the tau form below depends on c only through s^2.
  const float nab = al * rsqrtf(al) * (be * rsqrtf(be));   // sqrt(al) sqrt(be); NaN for a zero column: no rotation
  // largest relative inner product of the sweep (for the stopping rule)
  const float rel = __fdividef(fabsf(ga), nab);
  if (rel > rmax) rmax = rel;
  if (!(fabsf(ga) > tol * nab)) return false;
  const float zeta = __fdividef(be - al, 2.0f * ga);
  const float az = fabsf(zeta);
  const float q = fmaf(zeta, zeta, 1.0f);
  const float tt = az > 1e18f ? __fdividef(0.5f, zeta) : copysignf(__fdividef(1.0f, az + q * rsqrtf(q)), zeta);
  const float c = rsqrtf(fmaf(tt, tt, 1.0f));
  const float s = c * tt;
  const float tau = __fdividef(s, 1.0f + c);
#pragma unroll
  for (int u = 0; u < RP; ++u) {
    const float x = xm[u], y = ym[u];
    xm[u] = x - s * fmaf(tau, x, y);
    ym[u] = y + s * fmaf(-tau, y, x);
    if (WV) {
      const float vx = xv[u], vy = yv[u];
      xv[u] = vx - s * fmaf(tau, vx, vy);
      yv[u] = vy + s * fmaf(-tau, vy, vx);
    }
  }
  return true;
}

template <int RP, int GW, bool WV = true>
__device__ __forceinline__ void jc2_load(const float* __restrict__ col, int ls, int p, float (&m)[RP], float (&v)[RP]) {
#pragma unroll
  for (int u = 0; u < RP; ++u) {
    m[u] = col[p + 32 * GW * u];
    if (WV) v[u] = col[ls + p + 32 * GW * u];
  }
}

template <int RP, int GW, bool WV = true>
__device__ __forceinline__ void jc2_store(float* __restrict__ col, int ls, int p, const float (&m)[RP],
                                          const float (&v)[RP]) {
#pragma unroll
  for (int u = 0; u < RP; ++u) {
    col[p + 32 * GW * u] = m[u];
    if (WV) col[ls + p + 32 * GW * u] = v[u];
  }
}

constexpr int kJ2MaxL = 320;   // largest l of the pair kernel (16 CTAs x 2 blocks x 10 columns)
constexpr int kJUMaxL = 544;   // largest l of its M-only form (16 CTAs x 2 blocks x 17 columns)

// Physical buffers of cluster rank `rank` after e moves, four per CTA:
// top T, bottom B and the landing buffers FL / FR that blocks pushed by the
// left / right neighbour arrive in (-1: none).  A landing buffer is always
// the buffer this CTA last pushed to that same neighbour, so the neighbour
// can only write it after it has received (hence finished reading) it.
//   middle CTAs: (T, B, FL, FR) -> (FL, FR, B, T)
//   CTA 0:       T fixed, (B, FR) -> (FR, B)
//   last CTA:    (T, B, FL) -> (FL, T, B)   (its old top becomes its bottom in place)
__device__ __forceinline__ void jc5_bufs(int rank, int C, int e, int& t, int& b, int& fl, int& fr) {
  if (rank == 0) {
    t = 0;
    b = (e & 1) ? 2 : 1;
    fr = (e & 1) ? 1 : 2;
    fl = -1;
    return;
  }
  fr = -1;
  if (rank == C - 1) {
    const int m = e % 3;
    if (m == 0) { t = 0; b = 1; fl = 2; }
    else if (m == 1) { t = 2; b = 0; fl = 1; }
    else { t = 1; b = 2; fl = 0; }
    return;
  }
  switch (e & 3) {
    case 0: t = 0; b = 1; fl = 2; fr = 3; break;
    case 1: t = 2; b = 3; fl = 1; fr = 0; break;
    case 2: t = 1; b = 0; fl = 3; fr = 2; break;
    default: t = 3; b = 2; fl = 0; fr = 1; break;
  }
}

__device__ __forceinline__ uint32_t jc_smem_u32(const void* ptr) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}
__device__ __forceinline__ uint32_t jc_mapa(uint32_t saddr, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void jc_mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(jc_smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void jc_mbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(jc_smem_u32(bar)), "r"(bytes) : "memory");
}
// Bounded wait on a phase parity (`limit` SM clock cycles: about half a
// second by default); false when the limit expires.
__device__ __forceinline__ bool jc_mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (clock64() - t0 < limit) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(jc_smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
// Bulk copy of `bytes` from this CTA's shared memory into CTA `rank`'s, the
// arrival counted on that CTA's mbarrier (same offset in its shared memory).
__device__ __forceinline__ void jc_push(const float* src, float* dst_local_view, uint64_t* bar_local_view, int rank,
                                        uint32_t bytes) {
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          jc_mapa(jc_smem_u32(dst_local_view), rank)),
      "r"(jc_smem_u32(src)), "r"(bytes), "r"(jc_mapa(jc_smem_u32(bar_local_view), rank))
      : "memory");
}

// WV = false is the M-only form: the rotations are applied to M alone (no
// V_s is accumulated, a column is ls floats instead of 2 ls) and the
// epilogue writes the S2 outputs from M, for callers that form the right
// factor from B^T U_s Sigma^-1 (requires jb.r > 0).
template <int RP, int GW, bool WV = true>
__global__ void __launch_bounds__(640, 1)
jacobi_pair2_kernel(JacobiBatch jb, int l, int ls, int b, int max_sweeps, float tol, int* status) {
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int prob = blockIdx.x / C;
  float* __restrict__ Mg = jb.M[prob];
  float* __restrict__ Vg = jb.V[prob];
  extern __shared__ float4 jc2_smem4[];
  float* sm = reinterpret_cast<float*>(jc2_smem4);
  const int cs = WV ? 2 * ls : ls;            // floats per column: M part, then V part
  const int64_t bufsz = (int64_t)b * cs;      // floats per b-column buffer
  __shared__ float s_part[16][2][4];
  __shared__ int s_flags[16];
  __shared__ int s_ids[32];
  __shared__ int s_rmax;   // bits of the sweep's largest relative inner product (non-negative)
  __shared__ __align__(8) uint64_t rx_bar[2];   // incoming blocks of even / odd moves
  __shared__ float s_nrm[WV ? kJ2MaxL : kJUMaxL];  // column norms of the whole problem (rank-r outputs)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = warp / GW, wig = warp % GW, p = tid & (32 * GW - 1);
  const int nslots = 2 * C;

  if (tid < nslots) s_ids[tid] = tid;
  const uint32_t blk_bytes = static_cast<uint32_t>(bufsz * sizeof(float));
  const uint32_t rx_bytes = ((rank >= 1) + (rank <= C - 2)) * blk_bytes;
  if (tid == 0) {
    jc_mbar_init(&rx_bar[0]);
    jc_mbar_init(&rx_bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (C > 1) jc_mbar_expect(&rx_bar[0], rx_bytes);   // move 0
  }
  bool failed = false;
  int e_fail = -1;        // the move whose wait expired (this CTA)
  bool any_fail = false;  // some CTA of the cluster gave up (known to all after a sweep)
  for (int half = 0; half < 2; ++half) {
    float* buf = sm + half * bufsz;
    const int blk = 2 * rank + half;
    for (int64_t e = tid; e < bufsz; e += blockDim.x) {
      const int j = (int)(e / cs), i = (int)(e - (int64_t)j * cs);
      const int g = blk * b + j;
      float v = 0.f;
      if (g < l) {
        if (i < l) v = Mg[(int64_t)g * l + i];
        else if (WV && i >= ls && i - ls < l) v = (i - ls == g) ? 1.f : 0.f;
      }
      buf[e] = v;
    }
  }
  cluster.sync();

  const int be = b + (b & 1), half = be / 2, nreal = b / 2;
  int e = 0;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) s_rmax = 0;
    float rmax = 0.f;
    __syncthreads();
    for (int br = 0; br < 2 * C - 1; ++br) {
      int bt_, bb_, bfl, bfr;
      jc5_bufs(rank, C, e, bt_, bb_, bfl, bfr);
      float* topb = sm + bt_ * bufsz;
      float* botb = sm + bb_ * bufsz;
      if (br == 0) {  // pairs inside each block, circle method on b (+1 dummy) columns
        for (int t = 0; t < be - 1; ++t) {
          if (grp < 2 * nreal) {
            float* base = grp < nreal ? topb : botb;
            int q = grp < nreal ? grp : grp - nreal;
            int x = 0, y = 0;
            for (int k = 0; k < half; ++k) {
              int xx, yy;
              if (k == 0) {
                xx = 0;
                yy = 1 + t % (be - 1);
              } else {
                xx = 1 + (t + k) % (be - 1);
                yy = 1 + (t - k + (be - 1)) % (be - 1);
              }
              if (xx >= b || yy >= b) continue;
              if (q == 0) {
                x = xx;
                y = yy;
              }
              --q;
            }
            float xm[RP], xv[RP], ym[RP], yv[RP];
            float* cx = base + (int64_t)x * cs;
            float* cy = base + (int64_t)y * cs;
            jc2_load<RP, GW, WV>(cx, ls, p, xm, xv);
            jc2_load<RP, GW, WV>(cy, ls, p, ym, yv);
            if (jc2_rotate<RP, GW, WV>(xm, xv, ym, yv, tol, grp, wig, lane, s_part, rmax)) {
              jc2_store<RP, GW, WV>(cx, ls, p, xm, xv);
              jc2_store<RP, GW, WV>(cy, ls, p, ym, yv);
            }
          }
          __syncthreads();
        }
      }
      {  // top column grp against bottom column (grp + j) mod b, top held in registers
        float tm[RP], tv[RP];
        float* tcol = topb + (int64_t)grp * cs;
        jc2_load<RP, GW, WV>(tcol, ls, p, tm, tv);
        bool trot = false;
        for (int j = 0; j < b; ++j) {
          int k = grp + j;
          if (k >= b) k -= b;
          float* bcol = botb + (int64_t)k * cs;
          float bm[RP], bv[RP];
          jc2_load<RP, GW, WV>(bcol, ls, p, bm, bv);
          if (jc2_rotate<RP, GW, WV>(tm, tv, bm, bv, tol, grp, wig, lane, s_part, rmax)) {
            jc2_store<RP, GW, WV>(bcol, ls, p, bm, bv);
            trot = true;
          }
          __syncthreads();
        }
        if (trot) jc2_store<RP, GW, WV>(tcol, ls, p, tm, tv);
      }
      if (C > 1) {
        // Move: push the outgoing blocks into the neighbours' landing buffers
        // (bulk copies through distributed shared memory, counted on their
        // mbarriers) and wait for the incoming ones.  No cluster barrier.
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0 && !failed) {
          // after a timeout nothing more is armed, pushed or awaited: the
          // neighbours' waits expire in turn, the failure reaches every CTA
          // at the sweep's end, and each drains the copies issued into it
          jc_mbar_expect(&rx_bar[(e + 1) & 1], rx_bytes);   // next move; its previous phase is complete
          const bool drop = rank == jb.drop_rank && e == 0;   // failure-path tests only
          if (rank >= 1 && !drop) {  // bottom -> left neighbour's right landing buffer
            int t2, b2, l2, r2;
            jc5_bufs(rank - 1, C, e, t2, b2, l2, r2);
            jc_push(sm + bb_ * bufsz, sm + r2 * bufsz, &rx_bar[e & 1], rank - 1, blk_bytes);
          }
          if (rank <= C - 2 && !drop) {  // top (CTA 0: bottom) -> right neighbour's left landing buffer
            int t2, b2, l2, r2;
            jc5_bufs(rank + 1, C, e, t2, b2, l2, r2);
            jc_push(sm + (rank == 0 ? bb_ : bt_) * bufsz, sm + l2 * bufsz, &rx_bar[e & 1], rank + 1, blk_bytes);
          }
        }
        // block ids of the slots after this move, one slot per thread (read
        // here, written after the barrier below): slot 0 keeps its block,
        // slot 2 takes slot 1's, an even slot 2c >= 4 slot 2c - 2's, the
        // last slot 2C - 1 slot 2C - 2's, any other odd slot 2c + 1 slot 2c + 3's
        int nid = 0;
        if (tid < nslots) {
          const int src = tid == 0 ? 0 : tid == 2 ? 1 : (tid & 1) == 0 ? tid - 2 : tid == nslots - 1 ? nslots - 2 : tid + 2;
          nid = s_ids[src];
        }
        if (!failed && !jc_mbar_wait(&rx_bar[e & 1], (e >> 1) & 1, jb.wait_cycles)) {
          failed = true;
          set_status(status, LRAMM_ERR_TIMEOUT);
        }
        failed = __syncthreads_or(failed);   // one decision for the whole CTA
        if (failed && e_fail < 0) e_fail = e;
        if (tid < nslots) s_ids[tid] = nid;
        ++e;
      }
      __syncthreads();
    }
    // Convergence: the largest relative inner product |a.b| / (|a| |b|) met in
    // the sweep, over the cluster (one cluster barrier).  Below tol nothing
    // was rotated; below stopq tol the rotations of this sweep leave
    // inner products of the order of its square (quadratic convergence), so
    // a further sweep would rotate nothing: stop after this one.
    if (lane == 0) atomicMax(&s_rmax, __float_as_int(rmax));
    __syncthreads();
    // a CTA that gave up publishes INT_MAX: every CTA stops after this sweep
    if (tid < C) *cluster.map_shared_rank(&s_flags[rank], tid) = failed ? INT_MAX : s_rmax;
    cluster.sync();
    int mx = 0;
    for (int c = 0; c < C; ++c) mx = max(mx, s_flags[c]);
    if (mx == INT_MAX) {
      any_fail = true;
      break;
    }
    if (!(__int_as_float(mx) > jb.stopq * tol)) break;
  }
  if (!any_fail && sweep >= max_sweeps && tid == 0 && rank == 0) set_status(status, LRAMM_WARN_NOCONV);
  if (tid == 0 && rank == 0 && status) status[1 + jb.info0 + prob] = sweep < max_sweeps ? sweep + 1 : sweep;
  if (any_fail) {
    // Every push of every CTA was issued before the barrier above, and each
    // was aimed at a move phase its receiver had armed (a CTA arms a move's
    // phase one move ahead, and its neighbours stop pushing at most one move
    // after it stops).  A CTA whose wait expired drains the two phases it
    // left armed -- the move it gave up on and the next -- with bounded
    // waits, then the cluster barrier below: no bulk copy is still writing
    // into any CTA's shared memory when the CTAs go on (and exit).
    if (e_fail >= 0 && tid == 0)
      for (int mv = e_fail; mv <= e_fail + 1; ++mv) jc_mbar_wait(&rx_bar[mv & 1], (mv >> 1) & 1, jb.wait_cycles);
    __syncthreads();
  }
  // (a completed push needs no wait of its sender: each landed in a phase its
  // receiver awaited, which the sweep loop's waits or the drain above cover)
  cluster.sync();
  int bt_, bb_, bfl, bfr;
  jc5_bufs(rank, C, e, bt_, bb_, bfl, bfr);
  if (jb.r > 0) {
    // The sorted rank-r outputs straight from shared memory, as
    // svd_finalize_kernel forms them: column norms (same summation order),
    // shared with every CTA of the cluster, rank by descending norm (ties by
    // column index), the first r columns scaled and written.
    const FinalProb& fp = jb.fin[prob];
    const int r = jb.r;
    for (int hf = 0; hf < 2; ++hf) {
      const float* buf = sm + (hf == 0 ? bt_ : bb_) * bufsz;
      const int blk = s_ids[2 * rank + hf];
      for (int j = warp; j < b; j += (int)(blockDim.x >> 5)) {
        const int g = blk * b + j;
        const float* col = buf + (int64_t)j * cs;
        float sacc = 0.f;
        for (int i = lane; i < l; i += 32) sacc = fmaf(col[i], col[i], sacc);
        sacc = warp_sum(sacc);
        if (g < l && lane < C) *cluster.map_shared_rank(&s_nrm[g], lane) = sqrtf(sacc);
      }
    }
    cluster.sync();
    for (int hf = 0; hf < 2; ++hf) {
      const float* buf = sm + (hf == 0 ? bt_ : bb_) * bufsz;
      const int blk = s_ids[2 * rank + hf];
      for (int j = warp; j < b; j += (int)(blockDim.x >> 5)) {
        const int g = blk * b + j;
        if (g >= l) continue;
        const float v = s_nrm[g];
        int cnt = 0;
        for (int i = lane; i < l; i += 32) {
          const float u = s_nrm[i];
          cnt += (u > v) || (u == v && i < g);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        const int p = cnt;
        if (p >= r) continue;
        if (lane == 0) fp.sig[p] = v;
        const float inv = v > 0.f ? 1.0f / v : 0.f;
        const float u_scale = fp.s1_sigma ? 1.0f : inv;
        // M-only form: S2 = U_s Sigma^-1 (x sigma if s2_sigma) from M = U_s Sigma
        const float v_scale = WV ? (fp.s2_sigma ? v : 1.0f) : (fp.s2_sigma ? inv : inv * inv);
        const float* col = buf + (int64_t)j * cs;
        const int voff = WV ? ls : 0;
        for (int i = lane; i < l; i += 32) {
          const float o1 = col[i] * u_scale, o2 = col[voff + i] * v_scale;
          fp.S1[(int64_t)i * r + p] = o1;
          fp.S2[(int64_t)i * r + p] = o2;
          fp.S1T[(int64_t)p * l + i] = o1;
          fp.S2T[(int64_t)p * l + i] = o2;
        }
      }
    }
    return;
  }
  for (int hf = 0; hf < 2; ++hf) {
    const float* buf = sm + (hf == 0 ? bt_ : bb_) * bufsz;
    const int blk = s_ids[2 * rank + hf];
    for (int64_t q = tid; q < (int64_t)b * l; q += blockDim.x) {
      const int j = (int)(q / l), i = (int)(q - (int64_t)j * l);
      const int g = blk * b + j;
      if (g >= l) continue;
      const float* col = buf + (int64_t)j * cs;
      Mg[(int64_t)g * l + i] = col[i];
      if (WV) Vg[(int64_t)g * l + i] = col[ls + i];
    }
  }
}

// ---------------------------------------------------------------------------
// The pair kernel's rounds with the three-buffer moves, for 320 < l <= 544:
// one warp per column pair (b <= 17 warps), the top column held in
// registers for the b rounds of a block round, the three inner products in
// one shuffle tree and the fast rotation of jc2_rotate; the blocks circulate
// as in jacobi_cluster_kernel (three b-column buffers, pulls behind cluster
// barriers), since four buffers of b = 17 columns of M and V do not fit in
// shared memory.  Same schedule, threshold and stopping rule as the pair
// kernel.
// ---------------------------------------------------------------------------
template <int RP>
__global__ void __launch_bounds__(576)
jacobi_pair3_kernel(JacobiBatch jb, int l, int ls, int b, int max_sweeps, float tol, int* status) {
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int prob = blockIdx.x / C;
  float* __restrict__ Mg = jb.M[prob];
  float* __restrict__ Vg = jb.V[prob];
  extern __shared__ float4 jp3_smem4[];
  float* sm = reinterpret_cast<float*>(jp3_smem4);
  const int cs = 2 * ls;
  const int64_t bufsz = (int64_t)b * cs;
  __shared__ float s_part[16][2][4];
  __shared__ int s_flags[16];
  __shared__ int s_ids[32];
  __shared__ int s_rmax;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = warp, p = lane;
  const int nslots = 2 * C;

  if (tid < nslots) s_ids[tid] = tid;
  for (int half = 0; half < 2; ++half) {
    float* buf = sm + half * bufsz;
    const int blk = 2 * rank + half;
    for (int64_t e = tid; e < bufsz; e += blockDim.x) {
      const int j = (int)(e / cs), i = (int)(e - (int64_t)j * cs);
      const int g = blk * b + j;
      float v = 0.f;
      if (g < l) {
        if (i < l) v = Mg[(int64_t)g * l + i];
        else if (i >= ls && i - ls < l) v = (i - ls == g) ? 1.f : 0.f;
      }
      buf[e] = v;
    }
  }
  cluster.sync();

  const int be = b + (b & 1), half = be / 2, nreal = b / 2;
  int e = 0;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) s_rmax = 0;
    float rmax = 0.f;
    __syncthreads();
    for (int br = 0; br < 2 * C - 1; ++br) {
      int bt_, bb_, bf_;
      jc_bufs(rank, e, bt_, bb_, bf_);
      float* topb = sm + bt_ * bufsz;
      float* botb = sm + bb_ * bufsz;
      if (br == 0) {  // pairs inside each block, circle method on b (+1 dummy) columns
        for (int t = 0; t < be - 1; ++t) {
          if (grp < 2 * nreal) {
            float* base = grp < nreal ? topb : botb;
            int q = grp < nreal ? grp : grp - nreal;
            int x = 0, y = 0;
            for (int k = 0; k < half; ++k) {
              int xx, yy;
              if (k == 0) {
                xx = 0;
                yy = 1 + t % (be - 1);
              } else {
                xx = 1 + (t + k) % (be - 1);
                yy = 1 + (t - k + (be - 1)) % (be - 1);
              }
              if (xx >= b || yy >= b) continue;
              if (q == 0) {
                x = xx;
                y = yy;
              }
              --q;
            }
            float xm[RP], xv[RP], ym[RP], yv[RP];
            float* cx = base + (int64_t)x * cs;
            float* cy = base + (int64_t)y * cs;
            jc2_load<RP, 1>(cx, ls, p, xm, xv);
            jc2_load<RP, 1>(cy, ls, p, ym, yv);
            if (jc2_rotate<RP, 1>(xm, xv, ym, yv, tol, grp, 0, lane, s_part, rmax)) {
              jc2_store<RP, 1>(cx, ls, p, xm, xv);
              jc2_store<RP, 1>(cy, ls, p, ym, yv);
            }
          }
          __syncthreads();
        }
      }
      {  // top column grp against bottom column (grp + j) mod b, top held in registers
        float tm[RP], tv[RP];
        float* tcol = topb + (int64_t)grp * cs;
        jc2_load<RP, 1>(tcol, ls, p, tm, tv);
        bool trot = false;
        for (int j = 0; j < b; ++j) {
          int k = grp + j;
          if (k >= b) k -= b;
          float* bcol = botb + (int64_t)k * cs;
          float bm[RP], bv[RP];
          jc2_load<RP, 1>(bcol, ls, p, bm, bv);
          if (jc2_rotate<RP, 1>(tm, tv, bm, bv, tol, grp, 0, lane, s_part, rmax)) {
            jc2_store<RP, 1>(bcol, ls, p, bm, bv);
            trot = true;
          }
          __syncthreads();
        }
        if (trot) jc2_store<RP, 1>(tcol, ls, p, tm, tv);
      }
      if (C > 1) {
        cluster.sync();  // every CTA has finished rotating the blocks it is about to hand on
        // move 1: every CTA but 0 pulls its new top into its free buffer
        if (rank >= 1) {
          int st, sb, sf;
          jc_bufs(rank - 1, e, st, sb, sf);
          const float4* src =
              cluster.map_shared_rank(reinterpret_cast<float4*>(sm + (rank == 1 ? sb : st) * bufsz), rank - 1);
          float4* dst = reinterpret_cast<float4*>(sm + bf_ * bufsz);
          for (int64_t q = tid; q < bufsz / 4; q += blockDim.x) dst[q] = src[q];
        }
        cluster.sync();
        // move 2: every CTA but the last pulls its new bottom from the next CTA
        if (rank <= C - 2) {
          int st, sb, sf;
          jc_bufs(rank + 1, e, st, sb, sf);
          const float4* src = cluster.map_shared_rank(reinterpret_cast<float4*>(sm + sb * bufsz), rank + 1);
          float4* dst = reinterpret_cast<float4*>(sm + (rank == 0 ? bb_ : bt_) * bufsz);
          for (int64_t q = tid; q < bufsz / 4; q += blockDim.x) dst[q] = src[q];
        }
        if (tid == 0) {
          int nid[32];
          nid[0] = s_ids[0];
          nid[2] = s_ids[1];
          for (int c = 2; c < C; ++c) nid[2 * c] = s_ids[2 * c - 2];
          nid[2 * C - 1] = s_ids[2 * C - 2];
          for (int c = 0; c <= C - 2; ++c) nid[2 * c + 1] = s_ids[2 * c + 3];
          for (int q = 0; q < nslots; ++q) s_ids[q] = nid[q];
        }
        cluster.sync();
        ++e;
      } else {
        __syncthreads();
      }
    }
    if (lane == 0) atomicMax(&s_rmax, __float_as_int(rmax));
    __syncthreads();
    if (tid < C) *cluster.map_shared_rank(&s_flags[rank], tid) = s_rmax;
    cluster.sync();
    int mx = 0;
    for (int c = 0; c < C; ++c) mx = max(mx, s_flags[c]);
    cluster.sync();
    if (!(__int_as_float(mx) > jb.stopq * tol)) break;
  }
  if (sweep >= max_sweeps && tid == 0 && rank == 0) set_status(status, LRAMM_WARN_NOCONV);
  if (tid == 0 && rank == 0 && status) status[1 + jb.info0 + prob] = sweep < max_sweeps ? sweep + 1 : sweep;
  int bt_, bb_, bf_;
  jc_bufs(rank, e, bt_, bb_, bf_);
  for (int hf = 0; hf < 2; ++hf) {
    const float* buf = sm + (hf == 0 ? bt_ : bb_) * bufsz;
    const int blk = s_ids[2 * rank + hf];
    for (int64_t q = tid; q < (int64_t)b * l; q += blockDim.x) {
      const int j = (int)(q / l), i = (int)(q - (int64_t)j * l);
      const int g = blk * b + j;
      if (g >= l) continue;
      const float* col = buf + (int64_t)j * cs;
      Mg[(int64_t)g * l + i] = col[i];
      Vg[(int64_t)g * l + i] = col[ls + i];
    }
  }
}

// ---------------------------------------------------------------------------
// Opt-in shared memory per block on sm_100-class GPUs (227 KB), minus the
// static shared memory the kernels declare themselves.
static const int kSmemMax = 232448 - 1024;
// Warps per column pair of the cluster Jacobi (measured on GB300 at l = 272).
static const int kJacobiWarpsPerPair = 1;

lramm_status launch_chol(SmallBatch bt, int l, float shift_rel, int* status, cudaStream_t s) {
  const size_t smem = sizeof(float) * (size_t)l * (l + 1) / 2;
  if (smem > (size_t)kSmemMax) return LRAMM_ERR_UNSUPPORTED;
  LRAMM_CUDA_TRY(smem_cap(chol_kernel, (int)smem));
  chol_kernel<<<bt.n, 1024, smem, s>>>(bt, l, shift_rel, status);
  return last_launch();
}

lramm_status launch_trsm_rows(SmallBatch bt, int l, cudaStream_t s) {
  const int threads = 1024, nw = threads / 32;
  const size_t smem = sizeof(float) * ((size_t)l * (l + 1) / 2 + l + (size_t)nw * l);
  if (smem > (size_t)kSmemMax) return LRAMM_ERR_UNSUPPORTED;
  LRAMM_CUDA_TRY(smem_cap(trsm_rows_kernel, (int)smem));
  int64_t rows = 0;
  for (int i = 0; i < bt.n; ++i) rows = bt.p[i].rows > rows ? bt.p[i].rows : rows;
  int64_t grid = ceil_div(rows, nw);
  const int64_t cap = (num_sms() + bt.n - 1) / bt.n;
  if (grid > cap) grid = cap;
  trsm_rows_kernel<<<dim3((unsigned)grid, bt.n), threads, smem, s>>>(bt, l);
  return last_launch();
}

// Cluster size C and block width b for l columns: about 32 column pairs per
// CTA round (b <= 32 keeps one pair per warp), three b-column buffers of
// M and V per CTA within the shared-memory limit, at most 16 CTAs.
static bool jacobi_shape(int l, int& C, int& b, int& ls, size_t& smem) {
  ls = (int)round_up(l, 4);
  for (C = (int)ceil_div(l, 64); C <= 16; ++C) {
    if (C < 1) C = 1;
    b = (int)ceil_div(l, 2 * C);
    smem = sizeof(float) * 3 * (size_t)b * 2 * ls;
    if (smem <= (size_t)kSmemMax) return true;
  }
  return false;
}

int jacobi_max_l() {
  int best = 0;
  for (int l = 2; l <= 1024; ++l) {
    int C, b, ls;
    size_t smem;
    if (jacobi_shape(l, C, b, ls, smem)) best = l;
  }
  return best;
}

// Cluster shape: C = min(16, ceil(l/16)) CTAs, blocks of b columns, GW warps
// per column pair (64 b or 32 b threads), RP rows of a column per thread
// (columns zero padded to 32 GW RP rows).
static bool jacobi2_shape(int l, int gw, int& C, int& b, int& ls, int& rp, size_t& smem) {
  C = (int)ceil_div(l, 16);
  if (C < 1) C = 1;
  if (C > 16) C = 16;
  b = (int)ceil_div(l, 2 * C);
  rp = (int)ceil_div(l, 32 * gw);
  ls = 32 * gw * rp;
  smem = sizeof(float) * 4 * (size_t)b * 2 * ls;
  return b <= 10 && rp <= (gw == 2 ? 5 : 10) && smem <= (size_t)kSmemMax;
}

template <int RP, int GW>
static lramm_status launch_jacobi2_rp(JacobiBatch jb, int l, int ls, int C, int b, size_t smem, int max_sweeps,
                                      float tol, int* status, cudaStream_t s, bool& launched) {
  launched = false;
  auto kern = jacobi_pair2_kernel<RP, GW>;
  LRAMM_CUDA_TRY(smem_cap(kern, (int)smem));
  if (C > 8) LRAMM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(C * jb.n), 1, 1);
  cfg.blockDim = dim3((unsigned)(32 * GW * b), 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  LRAMM_CUDA_TRY(cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg));
  if (nclusters < 1) return LRAMM_OK;  // this cluster shape does not fit: caller falls back
  LRAMM_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, jb, l, ls, b, max_sweeps, tol, status));
  launched = true;
  return last_launch();
}

// The cluster Jacobi with gw warps per column pair (1 or 2); `done` is
// false when the shape is not available (the caller falls back).
lramm_status launch_jacobi_gw(JacobiBatch jb, int l, int gw, int max_sweeps, int* status, cudaStream_t s, bool& done) {
  done = false;
  int C2, b2, ls2, rp;
  size_t smem2;
  if (!jacobi2_shape(l, gw, C2, b2, ls2, rp, smem2)) return LRAMM_OK;
  const float tol2 = 4.0f * sqrtf((float)l) * 0x1p-24f;
#define JC_CASE(R, G) \
  case R: return launch_jacobi2_rp<R, G>(jb, l, ls2, C2, b2, smem2, max_sweeps, tol2, status, s, done);
  if (gw == 2) {
    switch (rp) {
      JC_CASE(1, 2) JC_CASE(2, 2) JC_CASE(3, 2) JC_CASE(4, 2) JC_CASE(5, 2)
      default: return LRAMM_OK;
    }
  }
  switch (rp) {
    JC_CASE(1, 1) JC_CASE(2, 1) JC_CASE(3, 1) JC_CASE(4, 1) JC_CASE(5, 1)
    JC_CASE(6, 1) JC_CASE(7, 1) JC_CASE(8, 1) JC_CASE(9, 1) JC_CASE(10, 1)
    default: return LRAMM_OK;
  }
#undef JC_CASE
}

// The pair-style three-buffer kernel: 16 CTAs, blocks of b = ceil(l / 32)
// columns (one warp each), RP = ceil(l / 32) rows per lane; `done` is false
// when the shape does not apply (l <= 320 or beyond 544) or does not fit.
template <int RP>
static lramm_status launch_pair3_rp(JacobiBatch jb, int l, int b, int max_sweeps, int* status, cudaStream_t s,
                                    bool& done) {
  const int C = 16, ls = 32 * RP;
  const size_t smem = sizeof(float) * 3 * (size_t)b * 2 * ls;
  if (smem > (size_t)kSmemMax || 32 * b > 576) return LRAMM_OK;
  auto kern = jacobi_pair3_kernel<RP>;
  LRAMM_CUDA_TRY(smem_cap(kern, (int)smem));
  LRAMM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(C * jb.n), 1, 1);
  cfg.blockDim = dim3((unsigned)(32 * b), 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  LRAMM_CUDA_TRY(cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg));
  if (nclusters < 1) return LRAMM_OK;
  const float tol = 4.0f * sqrtf((float)l) * 0x1p-24f;
  LRAMM_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, jb, l, ls, b, max_sweeps, tol, status));
  done = true;
  return last_launch();
}

lramm_status launch_jacobi_pair3(JacobiBatch jb, int l, int max_sweeps, int* status, cudaStream_t s, bool& done) {
  done = false;
  if (l <= kJ2MaxL || l > 544) return LRAMM_OK;
  const int b = (int)ceil_div(l, 32), rp = b;
  switch (rp) {
    case 11: return launch_pair3_rp<11>(jb, l, b, max_sweeps, status, s, done);
    case 12: return launch_pair3_rp<12>(jb, l, b, max_sweeps, status, s, done);
    case 13: return launch_pair3_rp<13>(jb, l, b, max_sweeps, status, s, done);
    case 14: return launch_pair3_rp<14>(jb, l, b, max_sweeps, status, s, done);
    case 15: return launch_pair3_rp<15>(jb, l, b, max_sweeps, status, s, done);
    case 16: return launch_pair3_rp<16>(jb, l, b, max_sweeps, status, s, done);
    case 17: return launch_pair3_rp<17>(jb, l, b, max_sweeps, status, s, done);
    default: return LRAMM_OK;
  }
}

// The M-only pair kernel: C = min(16, ceil(l / 16)) CTAs, blocks of
// b = ceil(l / 2C) <= 17 columns (one warp each), RP = ceil(l / 32) <= 17
// rows per lane, four b-column buffers of ls floats per column.
template <int RP>
static lramm_status launch_uonly_rp(JacobiBatch jb, int l, int C, int b, size_t smem, int max_sweeps, int* status,
                                    cudaStream_t s, bool check_only, bool& ok) {
  ok = false;
  const int ls = 32 * RP;
  auto kern = jacobi_pair2_kernel<RP, 1, false>;
  LRAMM_CUDA_TRY(smem_cap(kern, (int)smem));
  if (C > 8) LRAMM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(C * jb.n), 1, 1);
  cfg.blockDim = dim3((unsigned)(32 * b), 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  LRAMM_CUDA_TRY(cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg));
  if (nclusters < 1) return LRAMM_OK;
  ok = true;
  if (check_only) return LRAMM_OK;
  const float tol = 4.0f * sqrtf((float)l) * 0x1p-24f;
  LRAMM_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, jb, l, ls, b, max_sweeps, tol, status));
  return last_launch();
}

lramm_status launch_jacobi_uonly(JacobiBatch jb, int l, int max_sweeps, int* status, cudaStream_t s, bool check_only,
                                 bool& ok) {
  ok = false;
  if (l < 2 || l > kJUMaxL || jb.r <= 0 || jb.n < 1) return LRAMM_OK;
  // up to l = 192 wider blocks on fewer CTAs (fewer block moves per sweep;
  // l = 144: 6 CTAs of 12 columns, measured ahead of 9 of 8), beyond that
  // 16-column pairs per CTA (l = 272: 9 and 12 CTAs measured slower than 16)
  int C = (int)ceil_div(l, l <= 192 ? 24 : 16);
  if (C > 16) C = 16;
  const int b = (int)ceil_div(l, 2 * C), rp = (int)ceil_div(l, 32);
  const size_t smem = sizeof(float) * 4 * (size_t)b * 32 * rp;
  if (b > 17 || rp > 17 || smem > (size_t)kSmemMax) return LRAMM_OK;
#define JU_CASE(R) \
  case R: return launch_uonly_rp<R>(jb, l, C, b, smem, max_sweeps, status, s, check_only, ok);
  switch (rp) {
    JU_CASE(1) JU_CASE(2) JU_CASE(3) JU_CASE(4) JU_CASE(5) JU_CASE(6) JU_CASE(7) JU_CASE(8) JU_CASE(9)
    JU_CASE(10) JU_CASE(11) JU_CASE(12) JU_CASE(13) JU_CASE(14) JU_CASE(15) JU_CASE(16) JU_CASE(17)
    default: return LRAMM_OK;
  }
#undef JU_CASE
}

lramm_status launch_jacobi(JacobiBatch jb, int l, int max_sweeps, int* status, cudaStream_t s, bool* finalized) {
  *finalized = false;
  {
    bool done = false;
    LRAMM_TRY(launch_jacobi_gw(jb, l, kJacobiWarpsPerPair, max_sweeps, status, s, done));
    if (done) {
      *finalized = jb.r > 0;
      return LRAMM_OK;
    }
  }
  jb.r = 0;   // the three-buffer kernels leave M and V for svd_finalize
  {
    bool done = false;
    LRAMM_TRY(launch_jacobi_pair3(jb, l, max_sweeps, status, s, done));
    if (done) return LRAMM_OK;
  }
  int C, b, ls;
  size_t smem;
  if (!jacobi_shape(l, C, b, ls, smem)) return LRAMM_ERR_UNSUPPORTED;
  const float tol = 4.0f * sqrtf((float)l) * 0x1p-24f;
  LRAMM_CUDA_TRY(smem_cap(jacobi_cluster_kernel, (int)smem));
  if (C > 8)
    LRAMM_CUDA_TRY(cudaFuncSetAttribute(jacobi_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(C * jb.n), 1, 1);
  cfg.blockDim = dim3(1024, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  LRAMM_CUDA_TRY(cudaLaunchKernelEx(&cfg, jacobi_cluster_kernel, jb, l, ls, b, max_sweeps, tol, status));
  return last_launch();
}

lramm_status launch_svd_finalize(FinalBatch fb, int l, int r, cudaStream_t s) {
  const size_t smem = sizeof(float) * (2 * (size_t)l + (size_t)r);
  svd_finalize_kernel<<<dim3((unsigned)ceil_div(l, kFinRows), fb.n), 256, smem, s>>>(fb, l, r);
  return last_launch();
}


// ---------------------------------------------------------------------------
// Small helpers of the range-finder backward.
// out = the symmetric matrix holding M's lower triangle (diagonal included)
// on both sides: out[i][j] = M[max(i,j)][min(i,j)].
__global__ void copyltu_kernel(const float* __restrict__ M, float* __restrict__ out, int l) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)l * l;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / l), j = (int)(e - (int64_t)i * l);
    out[e] = i >= j ? M[e] : M[(int64_t)j * l + i];
  }
}
__global__ void identity_kernel(float* __restrict__ I, int l) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)l * l;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / l), j = (int)(e - (int64_t)i * l);
    I[e] = i == j ? 1.f : 0.f;
  }
}
__global__ void scale_kernel(float* __restrict__ x, int64_t n, float a) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    x[e] *= a;
}

__global__ void axpy_kernel(float* __restrict__ y, const float* __restrict__ x, int64_t n, float a) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = fmaf(a, x[e], y[e]);
}

static unsigned small_grid(int64_t n) {
  int64_t g = ceil_div(n, 256);
  return (unsigned)(g < 1 ? 1 : (g > 1216 ? 1216 : g));
}
lramm_status launch_copyltu(const float* M, float* out, int l, cudaStream_t s) {
  copyltu_kernel<<<small_grid((int64_t)l * l), 256, 0, s>>>(M, out, l);
  return last_launch();
}
lramm_status launch_identity(float* I, int l, cudaStream_t s) {
  identity_kernel<<<small_grid((int64_t)l * l), 256, 0, s>>>(I, l);
  return last_launch();
}
lramm_status launch_scale(float* x, int64_t n, float a, cudaStream_t s) {
  if (n <= 0) return LRAMM_OK;
  scale_kernel<<<small_grid(n), 256, 0, s>>>(x, n, a);
  return last_launch();
}

lramm_status launch_axpy(float* y, const float* x, int64_t n, float a, cudaStream_t s) {
  if (n <= 0) return LRAMM_OK;
  axpy_kernel<<<small_grid(n), 256, 0, s>>>(y, x, n, a);
  return last_launch();
}

}  // namespace lramm
