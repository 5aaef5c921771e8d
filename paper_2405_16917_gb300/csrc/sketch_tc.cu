// Products of an operand X with an l-column matrix on the 5th-generation
// tensor cores (tcgen05, sm_103a), TF32 inputs, FP32 accumulation:
//   a_mn = 0:  out = X   * B   (X rows x cols read K-major,  M = rows, K = cols)
//   a_mn = 1:  out = X^T * B   (X read in place MN-major,    M = cols, K = rows)
// B is K x l row-major (an MN-major operand), out M x l FP32 row-major.
// These are the sketch, power-iteration and projection products of the
// randomized range finder (Sec. 2.2, Algorithm 1's B = Q^* A): one pass over
// X each, so they are bound by HBM bandwidth.
//
// One CTA computes a 128-row block of out over a K range: a TMA producer
// warp streams 128 x 32 tiles of X and 32 x l tiles of B (128-byte swizzled)
// into a ring of shared-memory stages guarded by mbarriers, one thread of
// the MMA warp issues tcgen05.mma (M = 128, N <= 256 per instruction, two
// instructions when l > 256) into a TMEM accumulator, and four epilogue
// warps read TMEM back (tcgen05.ld) and store FP32 rows.  When the K range
// is split across CTAs, each writes a partial block and a reduction kernel
// adds the partials in a fixed order (deterministic results).
// Every mbarrier wait is bounded; on expiry the kernel latches
// LRAMM_ERR_TIMEOUT, stops issuing, waits (bounded) for its own copies and
// MMAs in flight, frees its TMEM and returns.
//
// BF16 operands X (sketch_bf_kernel): X is read as stored (BF16, exact
// tensor-core operands, kind::f16) and B is split once into BF16 parts
// B = B_hi + B_lo (B_hi = bf16(B), B_lo = bf16(B - B_hi), 16 significant
// bits together) with two MMAs per K step, or rounded to B_hi alone (one
// MMA, the LRAMM_SKETCH_BF16 arithmetic).  Stages of 32 K: X K-major with
// the 64-byte swizzle (a_mn = 0) or MN-major with the 128-byte swizzle
// (a_mn = 1), B parts MN-major with the 128-byte swizzle in 64-column
// chunks.  l > 512 (more than the 512 TMEM columns) is split into column
// blocks of at most 512, one grid slice each.
#include "tc_common.cuh"

namespace lramm {
namespace {

using namespace tc;

constexpr int kBM = 128;               // output rows per CTA = TMEM lanes
constexpr int kBK = 32;                // K per stage: 32 TF32 = one 128-byte swizzle row
constexpr int kAtom = 32;              // TF32 elements per 128-byte swizzle atom
constexpr int kThreads = 192;          // warp 0 TMA, warp 1 MMA, warps 2..5 epilogue
constexpr int kMaxStages = 8;

struct TcParams {
  int64_t M, K;
  int l, npad, n1, n2;
  int a_mn;
  int64_t kblocks;
  int kb_per_split;
  int stages;
  uint32_t a_bytes, b_bytes, tmem_cols;
  float* out;   // splits x M x l (or M x l when not split)
  int* status;
};

// Operand layouts:
//  * K-major: 128-byte swizzle (type 2), rows of 32 TF32 along K, 8-row
//    swizzle atoms 1024 bytes apart (SBO); a K step of 8 advances the start
//    address by 32 bytes inside the swizzled row.
//  * MN-major TF32: 128-byte swizzle with 32-byte atomicity (type 1, written
//    by TMA's SWIZZLE_128B_ATOM_32B): K rows of 32 MN elements, core
//    matrices 4 K rows tall (SBO = 512 bytes), 32-element MN atoms LBO
//    apart.  (The plain 128-byte swizzle reads as zeros for 32-bit MN-major
//    operands; measured on GB300.)
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t saddr) { return smem_desc(saddr, 16, 1024, 2); }
__device__ __forceinline__ uint64_t mnmajor_desc(uint32_t saddr) { return smem_desc(saddr, kAtom * kBK * 4, 512, 1); }

// Instruction descriptor of kind::tf32: D F32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), A / B major (bits 15, 16: 0 K-major, 1 MN-major),
// N >> 3 (bits 17-22), M >> 4 (bits 24-28).
__device__ __forceinline__ uint32_t idesc_tf32(int M, int N, int a_mn, int b_mn) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(a_mn) << 15) |
         (static_cast<uint32_t>(b_mn) << 16) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__global__ void __launch_bounds__(kThreads, 1)
sketch_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmB, TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + static_cast<size_t>(p.stages) * p.a_bytes;
  __shared__ __align__(8) uint64_t full_bar[kMaxStages], empty_bar[kMaxStages], tmem_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  volatile int* abort_flag = &abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * kBM;
  const int split = blockIdx.y;
  const int64_t kb0 = static_cast<int64_t>(split) * p.kb_per_split;
  const int64_t kb1 = min(p.kblocks, kb0 + p.kb_per_split);
  const int nkb = static_cast<int>(kb1 - kb0);

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&tmem_bar, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  const uint32_t tx_bytes = p.a_bytes + p.b_bytes;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    int issued = 0;
    bool ok = true;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % p.stages;
      if (i >= p.stages && !mbar_wait(&empty_bar[s], ((i / p.stages) & 1) ^ 1, abort_flag)) {
        ok = false;
        break;
      }
      mbar_expect_tx(&full_bar[s], tx_bytes);
      const int k0 = static_cast<int>((kb0 + i) * kBK);
      uint8_t* a_dst = sA + static_cast<size_t>(s) * p.a_bytes;
      if (p.a_mn) {
        for (int j = 0; j < kBM / kAtom; ++j)
          tma_load_2d(a_dst + j * (kAtom * kBK * 4), &tmX, &full_bar[s], static_cast<int>(m0) + j * kAtom, k0);
      } else {
        tma_load_2d(a_dst, &tmX, &full_bar[s], k0, static_cast<int>(m0));
      }
      uint8_t* b_dst = sB + static_cast<size_t>(s) * p.b_bytes;
      for (int j = 0; j < p.npad / kAtom; ++j)
        tma_load_2d(b_dst + j * (kAtom * kBK * 4), &tmB, &full_bar[s], j * kAtom, k0);
      ++issued;
    }
    if (!ok) {
      set_status(p.status, LRAMM_ERR_TIMEOUT);
      abort_sh = 1;
      // wait (bounded) for this CTA's copies still in flight
      const int first = issued > p.stages ? issued - p.stages : 0;
      for (int i = first; i < issued; ++i) {
        volatile int zero = 0;
        mbar_wait(&full_bar[i % p.stages], (i / p.stages) & 1, &zero);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    const int n1 = p.n1, n2 = p.n2;
    const uint32_t id1 = idesc_tf32(kBM, n1, p.a_mn, 1);
    const uint32_t id2 = n2 ? idesc_tf32(kBM, n2, p.a_mn, 1) : 0u;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % p.stages;
      if (!mbar_wait(&full_bar[s], (i / p.stages) & 1, abort_flag)) {
        set_status(p.status, LRAMM_ERR_TIMEOUT);
        abort_sh = 1;
        break;
      }
      tc_fence_after();
      const uint32_t a_base = smem_u32(sA + static_cast<size_t>(s) * p.a_bytes);
      const uint32_t b_base = smem_u32(sB + static_cast<size_t>(s) * p.b_bytes);
#pragma unroll
      for (int kk = 0; kk < kBK / 8; ++kk) {  // 8 TF32 (32 bytes) of K per instruction
        const uint64_t ad = p.a_mn ? mnmajor_desc(a_base + kk * 1024) : kmajor_desc(a_base + kk * 32);
        const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
        mma_tf32(tmem, ad, mnmajor_desc(b_base + kk * 1024), id1, acc);
        if (n2) mma_tf32(tmem + n1, ad, mnmajor_desc(b_base + (n1 / kAtom) * (kAtom * kBK * 4) + kk * 1024), id2, acc);
      }
      mma_commit(&empty_bar[s]);  // stage free once these MMAs have read it
    }
    mma_commit(&tmem_bar);        // accumulator complete (or every issued MMA done, on abort)
  } else if (warp >= 2) {
    // ---- epilogue: TMEM lanes 32q .. 32q+31 are rows m0 + 32q + lane
    const int q = warp & 3;
    volatile int zero = 0;  // wait for the MMAs even after an abort: they read shared memory
    const bool ok = mbar_wait(&tmem_bar, 0, &zero);
    tc_fence_after();
    const int64_t row = m0 + q * 32 + lane;
    float* dst = p.out + (static_cast<int64_t>(split) * p.M + row) * p.l;
    for (int c0 = 0; c0 < p.l; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(c0), v);
      if (!ok) continue;
      if (row < p.M) {
        const int nv = min(32, p.l - c0);  // multiple of 4
#pragma unroll
        for (int j = 0; j < 32; j += 4)
          if (j < nv) *reinterpret_cast<float4*>(dst + c0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
      }
    }
    if (!ok) set_status(p.status, LRAMM_ERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
  }
}

// ---------------------------------------------------------------------------
// BF16 X (see the file comment).
constexpr int kFK = 32;        // K per stage (BF16)
constexpr int kFAtom = 64;     // BF16 elements per 128-byte MN row
constexpr int kFChunk = kFAtom * kFK * 2;   // bytes of one 64-column x 32-K chunk

struct BfParams {
  int64_t M, K;
  int l, lout;          // columns of this launch's output block, row stride of out
  int npad;             // B parts' padded width (multiple of 64)
  int ncols, n1, n2;    // columns per CTA (<= 512), MMA widths (n1 <= 256)
  int nb;               // B parts: 1 (B_hi) or 2 (B_hi + B_lo)
  int a_mn;
  int64_t kblocks;
  int kb_per_split;
  int stages;
  uint32_t a_bytes, b_bytes, tmem_cols;
  float* out;
  int* status;
};

// K-major, 64-byte swizzle (layout type 4): rows of 32 BF16 along K, 8-row
// atoms 512 bytes apart; a K step of 16 advances 32 bytes in the row.
__device__ __forceinline__ uint64_t kmajor64_desc(uint32_t saddr) { return smem_desc(saddr, 16, 512, 4); }
// MN-major, 128-byte swizzle (type 2): K rows of 64 BF16 along MN, 8-row
// atoms 1024 bytes apart (SBO), 64-column chunks kFChunk bytes apart (LBO);
// a K step of 16 rows advances 2048 bytes.
__device__ __forceinline__ uint64_t mnmajor_bf_desc(uint32_t saddr) { return smem_desc(saddr, kFChunk, 1024, 2); }

__device__ __forceinline__ uint32_t idesc_bf(int M, int N, int a_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(a_mn) << 15) | (1u << 16) |
         (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__global__ void __launch_bounds__(kThreads, 1)
sketch_bf_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmBh,
                 const __grid_constant__ CUtensorMap tmBl, BfParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + static_cast<size_t>(p.stages) * p.a_bytes;
  __shared__ __align__(8) uint64_t full_bar[kMaxStages], empty_bar[kMaxStages], tmem_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  volatile int* abort_flag = &abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * kBM;
  const int split = blockIdx.y;
  const int c0 = blockIdx.z * p.ncols;              // first output column of this CTA
  const int ncols = min(p.ncols, p.l - c0);
  const int64_t kb0 = static_cast<int64_t>(split) * p.kb_per_split;
  const int64_t kb1 = min(p.kblocks, kb0 + p.kb_per_split);
  const int nkb = static_cast<int>(kb1 - kb0);
  const int nchunks = (ncols + kFAtom - 1) / kFAtom;
  const int n1 = ncols <= 256 ? ((ncols + 15) / 16) * 16 : 256;
  const int n2 = ncols <= 256 ? 0 : ((ncols - 256 + 15) / 16) * 16;

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&tmem_bar, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  const uint32_t part_bytes = static_cast<uint32_t>(nchunks) * kFChunk;   // one B part of one stage
  const uint32_t tx_bytes = p.a_bytes + static_cast<uint32_t>(p.nb) * part_bytes;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    int issued = 0;
    bool ok = true;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % p.stages;
      if (i >= p.stages && !mbar_wait(&empty_bar[s], ((i / p.stages) & 1) ^ 1, abort_flag)) {
        ok = false;
        break;
      }
      mbar_expect_tx(&full_bar[s], tx_bytes);
      const int k0 = static_cast<int>((kb0 + i) * kFK);
      uint8_t* a_dst = sA + static_cast<size_t>(s) * p.a_bytes;
      if (p.a_mn) {
        for (int j = 0; j < kBM / kFAtom; ++j)
          tma_load_2d(a_dst + j * kFChunk, &tmX, &full_bar[s], static_cast<int>(m0) + j * kFAtom, k0);
      } else {
        tma_load_2d(a_dst, &tmX, &full_bar[s], k0, static_cast<int>(m0));
      }
      uint8_t* b_dst = sB + static_cast<size_t>(s) * p.b_bytes;
      for (int j = 0; j < nchunks; ++j) {
        tma_load_2d(b_dst + j * kFChunk, &tmBh, &full_bar[s], c0 + j * kFAtom, k0);
        if (p.nb > 1) tma_load_2d(b_dst + part_bytes + j * kFChunk, &tmBl, &full_bar[s], c0 + j * kFAtom, k0);
      }
      ++issued;
    }
    if (!ok) {
      set_status(p.status, LRAMM_ERR_TIMEOUT);
      abort_sh = 1;
      const int first = issued > p.stages ? issued - p.stages : 0;
      for (int i = first; i < issued; ++i) {
        volatile int zero = 0;
        mbar_wait(&full_bar[i % p.stages], (i / p.stages) & 1, &zero);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    const uint32_t id1 = idesc_bf(kBM, n1, p.a_mn);
    const uint32_t id2 = n2 ? idesc_bf(kBM, n2, p.a_mn) : 0u;
    const uint32_t seg2 = static_cast<uint32_t>(256 / kFAtom) * kFChunk;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % p.stages;
      if (!mbar_wait(&full_bar[s], (i / p.stages) & 1, abort_flag)) {
        set_status(p.status, LRAMM_ERR_TIMEOUT);
        abort_sh = 1;
        break;
      }
      tc_fence_after();
      const uint32_t a_base = smem_u32(sA + static_cast<size_t>(s) * p.a_bytes);
      const uint32_t b_base = smem_u32(sB + static_cast<size_t>(s) * p.b_bytes);
#pragma unroll
      for (int kk = 0; kk < kFK / 16; ++kk) {  // 16 BF16 of K per instruction
        const uint64_t ad = p.a_mn ? mnmajor_bf_desc(a_base + kk * 2048) : kmajor64_desc(a_base + kk * 32);
        const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
        for (int b = 0; b < p.nb; ++b) {
          const uint32_t bb = b_base + b * part_bytes + kk * 2048;
          mma_bf(tmem, ad, mnmajor_bf_desc(bb), id1, (acc | b) ? 1u : 0u);
          if (n2) mma_bf(tmem + 256, ad, mnmajor_bf_desc(bb + seg2), id2, (acc | b) ? 1u : 0u);
        }
      }
      mma_commit(&empty_bar[s]);
    }
    mma_commit(&tmem_bar);
  } else if (warp >= 2) {
    // ---- epilogue: TMEM lanes 32q .. 32q+31 are rows m0 + 32q + lane
    const int q = warp & 3;
    volatile int zero = 0;
    const bool ok = mbar_wait(&tmem_bar, 0, &zero);
    tc_fence_after();
    const int64_t row = m0 + q * 32 + lane;
    float* dst = p.out + (static_cast<int64_t>(split) * p.M + row) * p.lout + c0;
    for (int cc = 0; cc < ncols; cc += 32) {
      float v[32];
      tmem_ld32(tmem + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(cc), v);
      if (!ok) continue;
      if (row < p.M) {
        const int nv = min(32, ncols - cc);  // multiple of 4
#pragma unroll
        for (int j = 0; j < 32; j += 4)
          if (j < nv) *reinterpret_cast<float4*>(dst + cc + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
      }
    }
    if (!ok) set_status(p.status, LRAMM_ERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
  }
}

// ---------------------------------------------------------------------------
// Q = Y L^-T on the tensor cores in split TF32: the CholeskyQR basis of the
// tensor-core range finders, a dense product with the explicit inverse in
// place of the panel triangular solve.  Y is rows x l (stride l); L^-1 comes
// as its TF32 high part Lh and low part Ll (l x l row-major, zero above the
// diagonal; Lh + Ll = L^-1 exactly in FP32); Q is rows x l and may be Y.
// Per K step of 8, three MMAs Yh Lh^T + Yl Lh^T + Yh Ll^T (FP32
// accumulation in TMEM, ~2^-21 relative, as the split-TF32 Gram); Y is
// split into Yh (in place) and Yl by the epilogue warps as each stage lands.
// Both operands are K-major with the 128-byte swizzle.  One CTA per 128
// rows reads all of its rows before its epilogue stores any (so Q = Y is
// safe); the output leaves as 32 x 32 blocks staged in the drained operand
// ring and written by TMA.  Waits are bounded as in sketch_tc_kernel.
// ---------------------------------------------------------------------------
struct BasisParams {
  int64_t rows;
  int l, n1, n2, nrows, nbox;   // MMA widths; rows of the L tiles (n1 + n2) and of one TMA box
  int kblocks, stages;
  uint32_t a_bytes, b_bytes, tmem_cols;   // one part of a Y tile (128 x 32) / of an L tile (nrows x 32)
  int* status;
};

__device__ __forceinline__ uint32_t idesc_tf32_kk(int M, int N) { return idesc_tf32(M, N, 0, 0); }

__global__ void __launch_bounds__(kThreads, 1)
basis_tc_kernel(const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmLh,
                const __grid_constant__ CUtensorMap tmLl, const __grid_constant__ CUtensorMap tmQ, BasisParams p,
                const int* __restrict__ cond) {
  if (cond && *cond == 0) return;   // predicated launch (the CholeskyQR fallback)
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[kMaxStages], split_bar[kMaxStages], empty_bar[kMaxStages], tmem_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  volatile int* abort_flag = &abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = static_cast<int64_t>(blockIdx.x) * kBM;
  const int nkb = p.kblocks;
  const uint32_t stage_bytes = 2 * p.a_bytes + 2 * p.b_bytes;   // Yh | Yl | Lh | Ll

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&split_bar[s], 128);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&tmem_bar, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: a 128 x 32 tile of Y and the nrows x 32 tiles of Lh, Ll per stage
    int issued = 0;
    bool ok = true;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % p.stages;
      if (i >= p.stages && !mbar_wait(&empty_bar[s], ((i / p.stages) & 1) ^ 1, abort_flag)) {
        ok = false;
        break;
      }
      mbar_expect_tx(&full_bar[s], p.a_bytes + 2 * p.b_bytes);
      const int k0 = i * kBK;
      uint8_t* st = smem + static_cast<size_t>(s) * stage_bytes;
      tma_load_2d(st, &tmY, &full_bar[s], k0, static_cast<int>(m0));
      for (int r0 = 0; r0 < p.nrows; r0 += p.nbox) {
        tma_load_2d(st + 2 * p.a_bytes + r0 * 128, &tmLh, &full_bar[s], k0, r0);
        tma_load_2d(st + 2 * p.a_bytes + p.b_bytes + r0 * 128, &tmLl, &full_bar[s], k0, r0);
      }
      ++issued;
    }
    if (!ok) {
      set_status(p.status, LRAMM_ERR_TIMEOUT);
      abort_sh = 1;
      const int first = issued > p.stages ? issued - p.stages : 0;
      for (int i = first; i < issued; ++i) {
        volatile int zero = 0;
        mbar_wait(&full_bar[i % p.stages], (i / p.stages) & 1, &zero);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    const uint32_t id2 = p.n2 ? idesc_tf32_kk(kBM, p.n2) : 0u;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % p.stages;
      if (!mbar_wait(&split_bar[s], (i / p.stages) & 1, abort_flag)) {
        set_status(p.status, LRAMM_ERR_TIMEOUT);
        abort_sh = 1;
        break;
      }
      tc_fence_after();
      const uint32_t yh = smem_u32(smem + static_cast<size_t>(s) * stage_bytes);
      const uint32_t yl = yh + p.a_bytes, lh = yh + 2 * p.a_bytes, ll = lh + p.b_bytes;
      // L^-1 is lower triangular: K block i (k0 = 32 i) meets only the
      // output columns n >= k0, so the first MMA group starts at column k0
      // (B rows k0 .., TMEM column k0) with N = n1 - k0; the first K block
      // covers (and initialises) every column
      const int k0 = i * kBK;
      const bool tri = k0 < p.n1;
      const uint32_t idt = tri ? idesc_tf32_kk(kBM, p.n1 - k0) : 0u;
      const uint32_t bo = static_cast<uint32_t>(k0) * 128;
#pragma unroll
      for (int kk = 0; kk < kBK / 8; ++kk) {   // 8 TF32 (32 bytes) of K per instruction
        const uint32_t ko = kk * 32;
        const uint32_t acc0 = (i > 0 || kk > 0) ? 1u : 0u;
        if (tri) {
          mma_tf32(tmem + k0, kmajor_desc(yh + ko), kmajor_desc(lh + bo + ko), idt, acc0);
          mma_tf32(tmem + k0, kmajor_desc(yl + ko), kmajor_desc(lh + bo + ko), idt, 1u);
          mma_tf32(tmem + k0, kmajor_desc(yh + ko), kmajor_desc(ll + bo + ko), idt, 1u);
        }
        if (p.n2) {   // L rows 256 .. : 256 rows of 128 bytes further on
          mma_tf32(tmem + 256, kmajor_desc(yh + ko), kmajor_desc(lh + 32768 + ko), id2, acc0);
          mma_tf32(tmem + 256, kmajor_desc(yl + ko), kmajor_desc(lh + 32768 + ko), id2, 1u);
          mma_tf32(tmem + 256, kmajor_desc(yh + ko), kmajor_desc(ll + 32768 + ko), id2, 1u);
        }
      }
      mma_commit(&empty_bar[s]);
    }
    mma_commit(&tmem_bar);
  } else if (warp >= 2) {
    // split each landed Y tile: high part in place, low part beside it
    // (element-wise, so the swizzled layout carries over)
    const int st = threadIdx.x - 64;   // 0 .. 127
    const int nq = static_cast<int>(p.a_bytes / 16);
    for (int i = 0; i < nkb; ++i) {
      const int s = i % p.stages;
      if (!mbar_wait(&full_bar[s], (i / p.stages) & 1, abort_flag)) {
        set_status(p.status, LRAMM_ERR_TIMEOUT);
        abort_sh = 1;
        break;
      }
      float4* h4 = reinterpret_cast<float4*>(smem + static_cast<size_t>(s) * stage_bytes);
      float4* l4 = reinterpret_cast<float4*>(smem + static_cast<size_t>(s) * stage_bytes + p.a_bytes);
      for (int e = st; e < nq; e += 128) {
        const float4 y = h4[e];
        float4 h;
        h.x = __uint_as_float(__float_as_uint(y.x) & 0xFFFFE000u);
        h.y = __uint_as_float(__float_as_uint(y.y) & 0xFFFFE000u);
        h.z = __uint_as_float(__float_as_uint(y.z) & 0xFFFFE000u);
        h.w = __uint_as_float(__float_as_uint(y.w) & 0xFFFFE000u);
        h4[e] = h;
        l4[e] = make_float4(y.x - h.x, y.y - h.y, y.z - h.z, y.w - h.w);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&split_bar[s])) : "memory");
    }
    // ---- epilogue: TMEM lanes 32q .. 32q+31 are rows m0 + 32q + lane.
    // Every copy into the ring was consumed by an MMA before tmem_bar
    // arrived, so the ring holds the staging blocks (two per warp).
    const int q = warp & 3;
    volatile int zero = 0;   // wait for the MMAs even after an abort: they read shared memory
    const bool ok = mbar_wait(&tmem_bar, 0, &zero);
    tc_fence_after();
    const int64_t rbase = m0 + q * 32;
    const uint32_t trow = tmem + (static_cast<uint32_t>(q * 32) << 16);
    for (int c0 = 0, nb = 0; c0 < p.l; c0 += 32, ++nb) {
      float v[32];
      tmem_ld32(trow + static_cast<uint32_t>(c0), v);
      float* stg = reinterpret_cast<float*>(smem) + (q * 2 + (nb & 1)) * 1024;
      if (nb >= 2) {   // this staging block's previous store has been read out
        if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        __syncwarp();
      }
#pragma unroll
      for (int c = 0; c < 8; ++c)
        *reinterpret_cast<float4*>(stg + lane * 32 + ((c ^ (lane & 7)) << 2)) =
            make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0 && ok && rbase < p.rows) {   // TMA clips the block at rows and l
        asm volatile(
            "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                reinterpret_cast<uint64_t>(&tmQ)),
            "r"(c0), "r"(static_cast<int>(rbase)), "r"(smem_u32(stg))
            : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
    }
    if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    __syncwarp();
    if (!ok) set_status(p.status, LRAMM_ERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
  }
}

// B (K x l FP32, row-major) -> B_hi, B_lo (K x npad BF16, zero padded).
__global__ void split_bf16_kernel(const float* __restrict__ B, int64_t K, int l, int npad, __nv_bfloat16* __restrict__ hi,
                                  __nv_bfloat16* __restrict__ lo) {
  const int64_t n = K * npad;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t k = e / npad;
    const int j = static_cast<int>(e - k * npad);
    const float b = j < l ? B[k * l + j] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(b);
    hi[e] = h;
    if (lo) lo[e] = __float2bfloat16_rn(b - __bfloat162float(h));
  }
}

// ---------------------------------------------------------------------------
// Gram G = Y^T Y of the CholeskyQR passes in split TF32 (three MMAs per K
// step): Y = Y_hi + Y_lo with Y_hi = Y truncated to TF32 (exactly
// representable) and Y_lo = Y - Y_hi (exact in FP32, 13 significant bits),
// G ~ Y_hi^T Y_hi + Y_hi^T Y_lo + Y_lo^T Y_hi (the dropped Y_lo^T Y_lo term
// and the TF32 rounding of Y_lo are ~2^-21 relative).  Both operands are
// MN-major views of the same staged K x W tiles (W = l rounded up to 128):
// the A operand of output row block mt is the tile's columns 128 mt ...
// TMA brings the FP32 tile of Y; warps 2..5 split it in shared memory into
// the high part (in place) and the low part (a second buffer of the same
// layout) before the MMAs of that stage, so Y is read once from memory.
// One CTA per (row block of G, K range), one launch per problem; split-K
// partials are added by split_reduce4_kernel.
//
// 128 < l <= 144: the rows 128 .. l-1 of G are the first tile's columns
// (transposed) except the corner block G[128.., 128..] (at most 16 x 16),
// which the converter warps accumulate in FP32 from a second, unswizzled TMA
// copy of those columns: one M tile of MMAs instead of two (the MMA issue
// is the kernel's clock), and a staged tile of ceil(l / 32) atoms.
constexpr int kGK = 16;   // rows of Y per Gram stage (16-row atoms: LBO 2 KB)
__device__ __forceinline__ uint64_t mnmajor_g_desc(uint32_t saddr) { return smem_desc(saddr, kAtom * kGK * 4, 512, 1); }

struct GramTcParams {
  int l, W, n1, n2;
  int mpc;       // M tiles per CTA: 2 when l <= 256 (both from one staged tile), else 1 (grid x = M tile)
  int corner;    // the corner width l - 128 when it is built in FP32 SIMT (then only tile 0 is MMA'd), else 0
  uint32_t cstride;   // bytes per stage of the corner copy (32 rows x corner FP32, 128-byte multiple)
  int nload;     // 32-column atoms loaded and split per stage: ceil(l / 32) (the rest only pad MMA reads)
  int64_t rows, kblocks;
  int kb_per_split;
  int stages;
  uint32_t part_bytes, tmem_cols;
  float* out;   // splits x l x l (or l x l when not split)
  int splits;
  int* status;
};

__global__ void __launch_bounds__(kThreads, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmC, GramTcParams p,
               const int* __restrict__ cond) {
  if (cond && *cond == 0) return;   // predicated launch (the CholeskyQR fallback)
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[kMaxStages], split_bar[kMaxStages], empty_bar[kMaxStages], tmem_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  volatile int* abort_flag = &abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = blockIdx.x, split = blockIdx.y;
  const int64_t kb0 = static_cast<int64_t>(split) * p.kb_per_split;
  const int64_t kb1 = min(p.kblocks, kb0 + p.kb_per_split);
  const int nkb = static_cast<int>(kb1 - kb0);   // >= 1: the host sizes the splits to the K range
  const uint32_t stage_bytes = 2 * p.part_bytes;

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&split_bar[s], 128);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&tmem_bar, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0 && lane == 0) {
    int issued = 0;
    bool ok = true;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % p.stages;
      if (i >= p.stages && !mbar_wait(&empty_bar[s], ((i / p.stages) & 1) ^ 1, abort_flag)) {
        ok = false;
        break;
      }
      mbar_expect_tx(&full_bar[s], static_cast<uint32_t>(p.nload) * (kAtom * kGK * 4) +
                                       static_cast<uint32_t>(p.corner) * (kGK * 4));
      const int k0 = static_cast<int>((kb0 + i) * kGK);
      uint8_t* dst = smem + static_cast<size_t>(s) * stage_bytes;
      for (int j = 0; j < p.nload; ++j) tma_load_2d(dst + j * (kAtom * kGK * 4), &tmY, &full_bar[s], j * kAtom, k0);
      if (p.corner)   // columns 128 .. l-1 of the same rows, row-major 32 x corner
        tma_load_2d(smem + static_cast<size_t>(p.stages) * stage_bytes + static_cast<size_t>(s) * p.cstride, &tmC,
                    &full_bar[s], kBM, k0);
      ++issued;
    }
    if (!ok) {
      set_status(p.status, LRAMM_ERR_TIMEOUT);
      abort_sh = 1;
      const int first = issued > p.stages ? issued - p.stages : 0;
      for (int i = first; i < issued; ++i) {
        volatile int zero = 0;
        mbar_wait(&full_bar[i % p.stages], (i / p.stages) & 1, &zero);
      }
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t id1 = idesc_tf32(kBM, p.n1, 1, 1);
    const uint32_t id1b = idesc_tf32(kBM, p.mpc == 2 ? ((p.l - kBM + 15) / 16) * 16 : 16, 1, 1);
    const uint32_t id2 = p.n2 ? idesc_tf32(kBM, p.n2, 1, 1) : 0u;
    const uint32_t seg2 = static_cast<uint32_t>(256 / kAtom) * (kAtom * kGK * 4);
    for (int i = 0; i < nkb; ++i) {
      const int s = i % p.stages;
      if (!mbar_wait(&split_bar[s], (i / p.stages) & 1, abort_flag)) {
        set_status(p.status, LRAMM_ERR_TIMEOUT);
        abort_sh = 1;
        break;
      }
      tc_fence_after();
      const uint32_t hi = smem_u32(smem + static_cast<size_t>(s) * stage_bytes);
      const uint32_t lo = hi + p.part_bytes;
      for (int t = 0; t < (p.corner ? 1 : p.mpc); ++t) {   // M tile mt + t into TMEM columns 256 t (n2 = 0 when mpc = 2)
        const uint32_t aoff = static_cast<uint32_t>((mt + t) * (kBM / kAtom)) * (kAtom * kGK * 4);
        const uint32_t d = tmem + static_cast<uint32_t>(t * 256);
        // with two tiles per CTA the second needs only columns 128 .. l-1
        // (its rows' columns 0 .. 127 are the first tile's, transposed)
        const uint32_t boff = t == 1 ? static_cast<uint32_t>(kBM / kAtom) * (kAtom * kGK * 4) : 0u;
        const uint32_t idt = t == 1 ? id1b : id1;
#pragma unroll
        for (int kk = 0; kk < kGK / 8; ++kk) {
          const uint32_t ko = kk * 1024;
          const uint32_t acc0 = (i > 0 || kk > 0) ? 1u : 0u;
          // (A, B) = (hi, hi), (hi, lo), (lo, hi)
          mma_tf32(d, mnmajor_g_desc(hi + aoff + ko), mnmajor_g_desc(hi + boff + ko), idt, acc0);
          mma_tf32(d, mnmajor_g_desc(hi + aoff + ko), mnmajor_g_desc(lo + boff + ko), idt, 1u);
          mma_tf32(d, mnmajor_g_desc(lo + aoff + ko), mnmajor_g_desc(hi + boff + ko), idt, 1u);
          if (p.n2) {
            mma_tf32(d + 256, mnmajor_g_desc(hi + aoff + ko), mnmajor_g_desc(hi + seg2 + ko), id2, acc0);
            mma_tf32(d + 256, mnmajor_g_desc(hi + aoff + ko), mnmajor_g_desc(lo + seg2 + ko), id2, 1u);
            mma_tf32(d + 256, mnmajor_g_desc(lo + aoff + ko), mnmajor_g_desc(hi + seg2 + ko), id2, 1u);
          }
        }
      }
      mma_commit(&empty_bar[s]);
    }
    mma_commit(&tmem_bar);
  } else if (warp >= 2) {
    // split each landed stage: high part in place, low part beside it
    const int st = threadIdx.x - 64;   // 0 .. 127
    const int nq = p.nload * (kAtom * kGK * 4 / 16);   // the loaded atoms (the rest only pad MMA reads)
    // the corner block: warp g = warp - 2 takes rows 4 g .. 4 g + 3 of each
    // stage, lane (bi, bj) = (lane / 8, lane mod 8) the 4 x 2 block at
    // corner rows 4 bi .., columns 2 bj .. (FP32 FMAs in row order)
    const int g = warp - 2, ci = 4 * (lane >> 3), cj = 2 * (lane & 7);
    const bool cown = ci < p.corner && cj < p.corner;
    const float* cbase = reinterpret_cast<const float*>(smem + static_cast<size_t>(p.stages) * stage_bytes);
    float cacc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int i = 0; i < nkb; ++i) {
      const int s = i % p.stages;
      if (!mbar_wait(&full_bar[s], (i / p.stages) & 1, abort_flag)) {
        set_status(p.status, LRAMM_ERR_TIMEOUT);
        abort_sh = 1;
        break;
      }
      float4* h4 = reinterpret_cast<float4*>(smem + static_cast<size_t>(s) * stage_bytes);
      float4* l4 = reinterpret_cast<float4*>(smem + static_cast<size_t>(s) * stage_bytes + p.part_bytes);
      for (int e = st; e < nq; e += 128) {
        const float4 y = h4[e];
        float4 h;
        h.x = __uint_as_float(__float_as_uint(y.x) & 0xFFFFE000u);
        h.y = __uint_as_float(__float_as_uint(y.y) & 0xFFFFE000u);
        h.z = __uint_as_float(__float_as_uint(y.z) & 0xFFFFE000u);
        h.w = __uint_as_float(__float_as_uint(y.w) & 0xFFFFE000u);
        h4[e] = h;
        l4[e] = make_float4(y.x - h.x, y.y - h.y, y.z - h.z, y.w - h.w);
      }
      if (cown) {   // before the arrival below: the stage (and its corner copy) is refilled only after it
        const float* cb = cbase + static_cast<size_t>(s) * (p.cstride / 4) + (kGK / 4 * g) * p.corner;
#pragma unroll
        for (int r = 0; r < kGK / 4; ++r) {
          const float4 a = *reinterpret_cast<const float4*>(cb + r * p.corner + ci);
          const float2 b = *reinterpret_cast<const float2*>(cb + r * p.corner + cj);
          cacc[0] = fmaf(a.x, b.x, cacc[0]);
          cacc[1] = fmaf(a.x, b.y, cacc[1]);
          cacc[2] = fmaf(a.y, b.x, cacc[2]);
          cacc[3] = fmaf(a.y, b.y, cacc[3]);
          cacc[4] = fmaf(a.z, b.x, cacc[4]);
          cacc[5] = fmaf(a.z, b.y, cacc[5]);
          cacc[6] = fmaf(a.w, b.x, cacc[6]);
          cacc[7] = fmaf(a.w, b.y, cacc[7]);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&split_bar[s])) : "memory");
    }
    const int q = warp & 3;
    volatile int zero = 0;
    const bool ok = mbar_wait(&tmem_bar, 0, &zero);
    tc_fence_after();
    float* gbase = p.out + static_cast<int64_t>(p.splits > 1 ? split : 0) * p.l * p.l;
    for (int t = 0; t < (p.corner ? 1 : p.mpc); ++t) {
      const int row = (mt + t) * kBM + q * 32 + lane;
      if ((mt + t) * kBM + q * 32 >= p.l) continue;   // this warp's TMEM lanes hold no row of G
      float* dst = gbase + static_cast<int64_t>(row) * p.l;
      // two tiles per CTA: the second tile's TMEM column j is G column 128 + j
      const int cfirst = (p.mpc == 2 && t == 1) ? kBM : 0;
      for (int c0 = cfirst; c0 < p.l; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(t * 256 + c0 - cfirst), v);
        if (!ok) continue;
        if (row < p.l) {
          const int nv = min(32, p.l - c0);
#pragma unroll
          for (int j = 0; j < 32; j += 4)
            if (j < nv) *reinterpret_cast<float4*>(dst + c0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
          if (p.mpc == 2 && t == 0 && c0 >= kBM) {   // G[c][row] = G[row][c], c >= 128: lanes write consecutive rows
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (j < nv) gbase[static_cast<int64_t>(c0 + j) * p.l + row] = v[j];
          }
        }
      }
    }
    if (p.corner) {
      // the four row groups' partial blocks, added in group order by warp 2
      // (every converter warp takes both barriers, also after an expired wait)
      float* red = reinterpret_cast<float*>(smem + static_cast<size_t>(p.stages) * (stage_bytes + p.cstride));
#pragma unroll
      for (int u = 0; u < 8; ++u) red[(g * 32 + lane) * 8 + u] = cacc[u];
      asm volatile("bar.sync 3, 128;" ::: "memory");
      if (g == 0 && ok && cown) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          float v = red[lane * 8 + u];
          v += red[(32 + lane) * 8 + u];
          v += red[(64 + lane) * 8 + u];
          v += red[(96 + lane) * 8 + u];
          const int a = ci + (u >> 1), b = cj + (u & 1);
          if (a < p.corner && b < p.corner) gbase[static_cast<int64_t>(kBM + a) * p.l + kBM + b] = v;
        }
      }
    }
    if (!ok) set_status(p.status, LRAMM_ERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
  }
}

// out = sum over splits of part[s] (fixed order), n4 float4 per split.
__global__ void split_reduce_kernel(const float4* __restrict__ part, int splits, int64_t n4, float4* __restrict__ out,
                                    const int* __restrict__ cond = nullptr) {
  if (cond && *cond == 0) return;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n4;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    float4 a = part[i];
    int s = 1;
    for (; s + 8 <= splits; s += 8) {   // eight loads in flight, added in split order
      float4 b[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) b[u] = part[static_cast<int64_t>(s + u) * n4 + i];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        a.x += b[u].x;
        a.y += b[u].y;
        a.z += b[u].z;
        a.w += b[u].w;
      }
    }
    for (; s < splits; ++s) {
      const float4 b = part[static_cast<int64_t>(s) * n4 + i];
      a.x += b.x;
      a.y += b.y;
      a.z += b.z;
      a.w += b.w;
    }
    out[i] = a;
  }
}

// The same sum for many splits and few outputs (the Gram partials): kRG
// threads per float4 of out, each adding its share of the splits in split
// order, then the kRG partial sums added in group order (deterministic, kRG
// times the loads in flight, and 256 / kRG outputs per CTA so that the grid
// covers the SMs).
constexpr int kRG = 16;
__global__ void __launch_bounds__(256) split_reduce4_kernel(const float4* __restrict__ part, int splits, int64_t n4,
                                                           float4* __restrict__ out, const int* __restrict__ cond) {
  if (cond && *cond == 0) return;
  constexpr int kOut = 256 / kRG;
  __shared__ float4 red[kRG][kOut];
  const int o = threadIdx.x % kOut, g = threadIdx.x / kOut;
  const int64_t i = blockIdx.x * static_cast<int64_t>(kOut) + o;
  const int per = (splits + kRG - 1) / kRG;
  const int s0 = g * per, s1 = min(splits, s0 + per);
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
  if (i < n4 && s0 < s1) {
    a = part[static_cast<int64_t>(s0) * n4 + i];
    int s = s0 + 1;
    for (; s + 4 <= s1; s += 4) {
      float4 b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) b[u] = part[static_cast<int64_t>(s + u) * n4 + i];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a.x += b[u].x;
        a.y += b[u].y;
        a.z += b[u].z;
        a.w += b[u].w;
      }
    }
    for (; s < s1; ++s) {
      const float4 b = part[static_cast<int64_t>(s) * n4 + i];
      a.x += b.x;
      a.y += b.y;
      a.z += b.z;
      a.w += b.w;
    }
  }
  red[g][o] = a;
  __syncthreads();
  if (g == 0 && i < n4) {
    float4 t = red[0][o];
    for (int q = 1; q < kRG; ++q) {
      if (q * per >= splits) break;   // groups past the last split are empty
      t.x += red[q][o].x;
      t.y += red[q][o].y;
      t.z += red[q][o].z;
      t.w += red[q][o].w;
    }
    out[i] = t;
  }
}

bool make_map_f32(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer, uint64_t row_bytes, uint32_t box_in,
                  uint32_t box_out, CUtensorMapSwizzle swizzle) {
  return make_map_2d(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, base, inner, outer, row_bytes, box_in, box_out, swizzle);
}

constexpr int kSmemBudget = 232448 - 2048;  // opt-in maximum minus alignment slack and static barriers

}  // namespace

bool sketch_tc_supported(int xbf, int64_t ldx, int l, const void* X, const void* B) {
  return !xbf && l % 4 == 0 && l >= 4 && l <= 512 && ldx % 4 == 0 && (reinterpret_cast<uintptr_t>(X) % 16) == 0 &&
         (reinterpret_cast<uintptr_t>(B) % 16) == 0;
}

// Split-K partials: one 128-row block per CTA slot (two slots per SM when l
// is narrow enough for two CTAs per SM).
// (workspace is sized at plan creation, before a device is known: for 152
// SMs; on a larger part the split count is capped by these buffers)
constexpr size_t kPartSlots = 152;
size_t sketch_tc_part_floats(int l) { return (l <= 160 ? 2 * kPartSlots : kPartSlots) * kBM * l; }

bool sketch_bf_supported(int64_t ldx, int l, const void* X, const void* B) {
  return l % 4 == 0 && l >= 4 && ldx % 8 == 0 && (reinterpret_cast<uintptr_t>(X) % 16) == 0 &&
         (reinterpret_cast<uintptr_t>(B) % 16) == 0;
}

size_t sketch_bf_split_bytes(int64_t K, int l) { return 2 * sizeof(__nv_bfloat16) * K * round_up(l, kFAtom) + 256; }

lramm_status sketch_bf(int a_mn, const void* X, int64_t rows, int64_t cols, int64_t ldx, const float* B, int l,
                       int nb, float* out, float* part, size_t part_floats, void* split, size_t split_bytes,
                       int* status, cudaStream_t s) {
  if (!sketch_bf_supported(ldx, l, X, B) || (nb != 1 && nb != 2)) return LRAMM_ERR_UNSUPPORTED;
  const int64_t M = a_mn ? cols : rows, K = a_mn ? rows : cols;
  if (M <= 0 || K <= 0) return LRAMM_OK;
  if (M > INT32_MAX || K > INT32_MAX) return LRAMM_ERR_UNSUPPORTED;
  if (split_bytes < sketch_bf_split_bytes(K, l)) return LRAMM_ERR_WORKSPACE;
  BfParams p{};
  p.M = M;
  p.K = K;
  p.l = l;
  p.lout = l;
  p.npad = static_cast<int>(round_up(l, kFAtom));
  const int nslices = static_cast<int>(ceil_div(l, 512));
  p.ncols = static_cast<int>(round_up(ceil_div(l, nslices), kFAtom));   // multiple of 64, <= 512
  p.nb = nb;
  p.a_mn = a_mn;
  p.kblocks = ceil_div(K, kFK);
  p.a_bytes = kBM * kFK * 2;
  p.b_bytes = static_cast<uint32_t>(nb) * static_cast<uint32_t>(p.ncols / kFAtom) * kFChunk;
  p.stages = static_cast<int>((kSmemBudget - 1024) / (p.a_bytes + p.b_bytes));
  if (p.stages > kMaxStages) p.stages = kMaxStages;
  if (p.stages < 2) return LRAMM_ERR_UNSUPPORTED;
  uint32_t tc = 32;
  while (tc < static_cast<uint32_t>(p.ncols)) tc <<= 1;
  p.tmem_cols = tc;
  p.status = status;
  const int64_t mtiles = ceil_div(M, kBM);
  int64_t splits = num_sms() / (mtiles * nslices);
  if (splits > p.kblocks / 8) splits = p.kblocks / 8;
  if (splits < 1) splits = 1;
  while (splits > 1 && static_cast<size_t>(splits) * M * l > part_floats) --splits;
  p.kb_per_split = static_cast<int>(ceil_div(p.kblocks, splits));
  splits = ceil_div(p.kblocks, p.kb_per_split);
  p.out = splits > 1 ? part : out;

  // B parts (K x npad BF16 each)
  __nv_bfloat16* hi = reinterpret_cast<__nv_bfloat16*>((reinterpret_cast<uintptr_t>(split) + 255) & ~uintptr_t(255));
  __nv_bfloat16* lo = nb > 1 ? hi + K * p.npad : nullptr;
  {
    int64_t g = ceil_div(K * p.npad, 256);
    if (g > num_sms() * 8) g = num_sms() * 8;
    split_bf16_kernel<<<static_cast<unsigned>(g), 256, 0, s>>>(B, K, l, p.npad, hi, lo);
    LRAMM_TRY(last_launch());
  }
  CUtensorMap mX, mBh, mBl;
  if (!make_map_2d(&mX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, X, cols, rows, ldx * 2, a_mn ? kFAtom : kFK,
                   a_mn ? kFK : kBM, a_mn ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B))
    return LRAMM_ERR_CUDA;
  if (!make_map_2d(&mBh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, hi, p.npad, K, static_cast<uint64_t>(p.npad) * 2, kFAtom,
                   kFK, CU_TENSOR_MAP_SWIZZLE_128B))
    return LRAMM_ERR_CUDA;
  if (!make_map_2d(&mBl, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, nb > 1 ? lo : hi, p.npad, K,
                   static_cast<uint64_t>(p.npad) * 2, kFAtom, kFK, CU_TENSOR_MAP_SWIZZLE_128B))
    return LRAMM_ERR_CUDA;
  const size_t smem = 1024 + static_cast<size_t>(p.stages) * (p.a_bytes + p.b_bytes);
  LRAMM_CUDA_TRY(smem_cap(sketch_bf_kernel, (int)smem));
  sketch_bf_kernel<<<dim3(static_cast<unsigned>(mtiles), static_cast<unsigned>(splits), static_cast<unsigned>(nslices)),
                     kThreads, smem, s>>>(mX, mBh, mBl, p);
  LRAMM_TRY(last_launch());
  if (splits > 1) {
    const int64_t n4 = M * l / 4;
    int64_t g = ceil_div(n4, 256);
    if (g > num_sms() * 8) g = num_sms() * 8;
    split_reduce_kernel<<<static_cast<unsigned>(g), 256, 0, s>>>(reinterpret_cast<const float4*>(part),
                                                                  static_cast<int>(splits), n4,
                                                                  reinterpret_cast<float4*>(out));
    LRAMM_TRY(last_launch());
  }
  return LRAMM_OK;
}

lramm_status sketch_tc(int a_mn, const void* X, int64_t rows, int64_t cols, int64_t ldx, int xbf, const float* B,
                       int l, float* out, float* part, size_t part_floats, int* status, cudaStream_t s) {
  if (!sketch_tc_supported(xbf, ldx, l, X, B)) return LRAMM_ERR_UNSUPPORTED;
  const int64_t M = a_mn ? cols : rows, K = a_mn ? rows : cols;
  if (M <= 0 || K <= 0) return LRAMM_OK;
  if (M > INT32_MAX || K > INT32_MAX) return LRAMM_ERR_UNSUPPORTED;
  TcParams p{};
  p.M = M;
  p.K = K;
  p.l = l;
  p.npad = static_cast<int>(round_up(l, kAtom));
  p.n1 = l <= 256 ? static_cast<int>(round_up(l, 16)) : 256;
  p.n2 = l <= 256 ? 0 : static_cast<int>(round_up(l - 256, 16));
  p.a_mn = a_mn;
  p.kblocks = ceil_div(K, kBK);
  p.a_bytes = kBM * kBK * 4;
  p.b_bytes = static_cast<uint32_t>(p.npad) * kBK * 4;
  // Two CTAs per SM when a three-stage ring fits in half the shared memory
  // (l <= ~160): one CTA's epilogue and ramp-up overlap the other's stream
  // (measured 1.4x faster on the 32768 x 4096 products); otherwise one CTA
  // per SM with the deepest ring that fits.
  const uint32_t stage_bytes = p.a_bytes + p.b_bytes;
  const int nsm = num_sms();
  int slots = nsm;
  if (1024 + 3 * stage_bytes <= 112 * 1024) {   // two CTAs within the SM's 228 KB
    p.stages = 3;
    slots = 2 * nsm;
  } else {
    p.stages = static_cast<int>((kSmemBudget - 1024) / stage_bytes);
    if (p.stages > kMaxStages) p.stages = kMaxStages;
  }
  if (p.stages < 2) return LRAMM_ERR_UNSUPPORTED;
  uint32_t tc = 32;
  while (tc < static_cast<uint32_t>(p.n1 + p.n2)) tc <<= 1;
  p.tmem_cols = tc;
  p.status = status;
  const int64_t mtiles = ceil_div(M, kBM);
  int64_t splits = slots / mtiles;
  if (splits > p.kblocks / 4) splits = p.kblocks / 4;
  if (splits < 1) splits = 1;
  while (splits > 1 && static_cast<size_t>(splits) * M * l > part_floats) --splits;
  p.kb_per_split = static_cast<int>(ceil_div(p.kblocks, splits));
  splits = ceil_div(p.kblocks, p.kb_per_split);
  p.out = splits > 1 ? part : out;

  CUtensorMap mX, mB;
  if (!make_map_f32(&mX, X, cols, rows, ldx * 4, kAtom, a_mn ? kBK : kBM,
                    a_mn ? CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B : CU_TENSOR_MAP_SWIZZLE_128B))
    return LRAMM_ERR_CUDA;
  if (!make_map_f32(&mB, B, l, K, static_cast<uint64_t>(l) * 4, kAtom, kBK, CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B))
    return LRAMM_ERR_CUDA;
  const size_t smem = 1024 + static_cast<size_t>(p.stages) * (p.a_bytes + p.b_bytes);
  LRAMM_CUDA_TRY(smem_cap(sketch_tc_kernel, (int)smem));
  sketch_tc_kernel<<<dim3(static_cast<unsigned>(mtiles), static_cast<unsigned>(splits)), kThreads, smem, s>>>(mX, mB, p);
  LRAMM_TRY(last_launch());
  if (splits > 1) {
    const int64_t n4 = M * l / 4;
    int64_t g = ceil_div(n4, 256);
    if (g > num_sms() * 8) g = num_sms() * 8;
    split_reduce_kernel<<<static_cast<unsigned>(g), 256, 0, s>>>(reinterpret_cast<const float4*>(part),
                                                                  static_cast<int>(splits), n4,
                                                                  reinterpret_cast<float4*>(out));
    LRAMM_TRY(last_launch());
  }
  return LRAMM_OK;
}

// Gram on the tensor cores (split TF32) for one or two problems.
constexpr size_t kGramCoSmem = 112 * 1024;
static int gram_tc_width(int l) { return static_cast<int>(round_up(l, kBM)); }   // staged tile width
size_t gram_tc_part_floats(int l) { return kPartSlots * l * l; }

bool gram_tc_supported(int l) { return l >= 4 && l % 4 == 0 && l <= 512; }

lramm_status gram_tc(int n, const float* const* Y, const int64_t* rows, float* const* G, int l, float* part,
                     size_t part_floats, int* status, cudaStream_t s, const int* cond) {
  if (!gram_tc_supported(l) || n < 1 || n > 2) return LRAMM_ERR_UNSUPPORTED;
  GramTcParams p{};
  p.l = l;
  p.W = gram_tc_width(l);
  p.n1 = l <= 256 ? static_cast<int>(round_up(l, 16)) : 256;
  p.n2 = l <= 256 ? 0 : static_cast<int>(round_up(l - 256, 16));
  const int mtiles = static_cast<int>(ceil_div(l, kBM));
  // l <= 256: one CTA issues both M tiles' MMAs from each staged tile (the
  // tile is loaded and split once), accumulators at TMEM columns 0 and 256;
  // l <= 144: the second tile's only new block is the corner, in FP32 SIMT
  p.mpc = (mtiles == 2 && p.n2 == 0) ? 2 : 1;
  p.corner = (p.mpc == 2 && l - kBM <= 16) ? l - kBM : 0;
  p.nload = static_cast<int>(ceil_div(l, kAtom));
  if (p.corner) p.W = p.nload * kAtom;   // tile 0's A (atoms 0..3) and B (n1 columns) lie within the loaded atoms
  p.part_bytes = static_cast<uint32_t>(p.W) * kGK * 4;
  p.cstride = p.corner ? static_cast<uint32_t>(round_up(static_cast<size_t>(kGK) * p.corner * 4, 128)) : 0u;
  const size_t red_bytes = p.corner ? 4 * 32 * 8 * sizeof(float) : 0;
  // at most ~110 KB when that still holds four stages: the CTA then fits
  // beside one CTA of a concurrent range-finder product on its SM
  const size_t gstage = 2 * static_cast<size_t>(p.part_bytes) + p.cstride;
  p.stages = static_cast<int>((kGramCoSmem - 1024 - red_bytes) / gstage);
  if (p.stages < 4) p.stages = static_cast<int>((kSmemBudget - 1024 - red_bytes) / gstage);
  if (p.stages > kMaxStages) p.stages = kMaxStages;
  if (p.stages < 2) return LRAMM_ERR_UNSUPPORTED;
  uint32_t tc = 32;
  while (tc < static_cast<uint32_t>(p.n1 + p.n2)) tc <<= 1;
  p.tmem_cols = (p.mpc == 2 && !p.corner) ? 512u : tc;
  p.status = status;
  const int gx = mtiles / p.mpc;
  const size_t smem = 1024 + static_cast<size_t>(p.stages) * (2 * p.part_bytes + p.cstride) + red_bytes;
  LRAMM_CUDA_TRY(smem_cap(gram_tc_kernel, (int)smem));
  for (int i = 0; i < n; ++i) {
    if (rows[i] < 1) return LRAMM_ERR_INVALID_ARG;
    p.rows = rows[i];
    p.kblocks = ceil_div(rows[i], kGK);
    int64_t splits = num_sms() / (p.mpc == 2 ? 1 : mtiles);
    if (splits > p.kblocks / 2) splits = p.kblocks / 2;   // at least two K blocks per CTA
    if (splits < 1) splits = 1;
    while (splits > 1 && static_cast<size_t>(splits) * l * l > part_floats) --splits;
    p.kb_per_split = static_cast<int>(ceil_div(p.kblocks, splits));
    splits = ceil_div(p.kblocks, p.kb_per_split);   // every CTA has at least one K block
    p.splits = static_cast<int>(splits);
    p.out = splits > 1 ? part : G[i];
    // the FP32 rows of Y (l % 4 == 0: 16-byte row pitch); tile atoms beyond
    // l and rows beyond the end are loaded out of range (x a multiple of 32)
    // and arrive as zeros
    CUtensorMap my, mc;
    if (!make_map_f32(&my, Y[i], l, rows[i], static_cast<uint64_t>(l) * 4, kAtom, kGK,
                      CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B))
      return LRAMM_ERR_CUDA;
    if (p.corner) {   // the corner columns 128 .. l-1, a dense 32 x corner box (corner * 4 bytes: a multiple of 16)
      if (!make_map_f32(&mc, Y[i], l, rows[i], static_cast<uint64_t>(l) * 4, static_cast<uint32_t>(p.corner), kGK,
                        CU_TENSOR_MAP_SWIZZLE_NONE))
        return LRAMM_ERR_CUDA;
    } else {
      mc = my;   // not read
    }
    gram_tc_kernel<<<dim3(static_cast<unsigned>(gx), static_cast<unsigned>(splits)), kThreads, smem, s>>>(my, mc, p,
                                                                                                        cond);
    LRAMM_TRY(last_launch());
    if (splits > 1) {
      const int64_t n4 = static_cast<int64_t>(l) * l / 4;
      split_reduce4_kernel<<<static_cast<unsigned>(ceil_div(n4, 256 / kRG)), 256, 0, s>>>(
          reinterpret_cast<const float4*>(part), static_cast<int>(splits), n4, reinterpret_cast<float4*>(G[i]), cond);
      LRAMM_TRY(last_launch());
    }
  }
  return LRAMM_OK;
}

// Q = Y L^-T in split TF32 from the inverse's parts (see basis_tc_kernel).
bool basis_tc_supported(int l) { return l >= 16 && l % 4 == 0 && l <= 288; }

lramm_status basis_tc(const float* Y, int64_t rows, const float* Lh, const float* Ll, float* Q, int l, int* status,
                      cudaStream_t s, const int* cond) {
  if (!basis_tc_supported(l)) return LRAMM_ERR_UNSUPPORTED;
  if (rows <= 0) return LRAMM_OK;
  if (rows > INT32_MAX) return LRAMM_ERR_UNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(Y) | reinterpret_cast<uintptr_t>(Lh) | reinterpret_cast<uintptr_t>(Ll) |
       reinterpret_cast<uintptr_t>(Q)) & 15)
    return LRAMM_ERR_UNSUPPORTED;
  BasisParams p{};
  p.rows = rows;
  p.l = l;
  p.n1 = l <= 256 ? static_cast<int>(round_up(l, 16)) : 256;
  p.n2 = l <= 256 ? 0 : static_cast<int>(round_up(l - 256, 16));
  p.nrows = p.n1 + p.n2;
  p.nbox = p.nrows <= 256 ? p.nrows : p.nrows / 2;   // a multiple of 8, at most 256
  p.kblocks = static_cast<int>(ceil_div(l, kBK));
  p.a_bytes = kBM * kBK * 4;
  p.b_bytes = static_cast<uint32_t>(p.nrows) * kBK * 4;
  const uint32_t stage = 2 * p.a_bytes + 2 * p.b_bytes;
  int st = static_cast<int>((kSmemBudget - 1024) / stage);
  if (st > kMaxStages) st = kMaxStages;
  if (st > p.kblocks) st = p.kblocks;
  if (st < 1 || (st < 2 && p.kblocks > 1)) return LRAMM_ERR_UNSUPPORTED;
  p.stages = st;
  uint32_t tc = 32;
  while (tc < static_cast<uint32_t>(p.n1 + p.n2 + (p.n2 ? 256 - p.n1 : 0))) tc <<= 1;
  p.tmem_cols = tc;
  p.status = status;
  CUtensorMap mY, mLh, mLl, mQ;
  const uint64_t pitch = static_cast<uint64_t>(l) * 4;
  if (!make_map_f32(&mY, Y, l, rows, pitch, kAtom, kBM, CU_TENSOR_MAP_SWIZZLE_128B) ||
      !make_map_f32(&mLh, Lh, l, l, pitch, kAtom, p.nbox, CU_TENSOR_MAP_SWIZZLE_128B) ||
      !make_map_f32(&mLl, Ll, l, l, pitch, kAtom, p.nbox, CU_TENSOR_MAP_SWIZZLE_128B) ||
      !make_map_f32(&mQ, Q, l, rows, pitch, kAtom, 32, CU_TENSOR_MAP_SWIZZLE_128B))
    return LRAMM_ERR_CUDA;
  const size_t smem = 1024 + static_cast<size_t>(p.stages) * stage;
  LRAMM_CUDA_TRY(smem_cap(basis_tc_kernel, (int)smem));
  basis_tc_kernel<<<static_cast<unsigned>(ceil_div(rows, kBM)), kThreads, smem, s>>>(mY, mLh, mLl, mQ, p, cond);
  return last_launch();
}

}  // namespace lramm
