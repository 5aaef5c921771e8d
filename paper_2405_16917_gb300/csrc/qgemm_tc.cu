// Products on the 5th-generation tensor cores, FP32 accumulation in TMEM:
//
//   acc[i][j] = sum_k L[i][k] R[j][k]      (L: M x K, R: N x K, both K-major)
//
// in three operand kinds:
//  * BF16 codes (INT8 factors of Algorithm 2 / 3): every integer of
//    magnitude <= 127 is exact in BF16; tcgen05.mma kind::f16.  A product
//    of two codes is at most 127^2 = 16129, so a sum of at most 1024 of
//    them stays below 2^24: each CTA sums at most 1024 products (16 K blocks
//    of 64), its accumulator holds the exact integer, and longer K is split
//    across CTAs whose partials are added as 32-bit integers.
//  * FP8 e4m3 codes (E4M3 factors, and INT4 factors, whose integer codes
//    |c| <= 7 are exact e4m3 values); kind::f8f6f4.  INT4 sums are exact
//    (|sum| <= 49 K < 2^24 for K < 342,000); e4m3 sums are FP32 sums.
//  * FP32 operands as TF32 (the dense products of the range-finder
//    backward); kind::tf32, no scales.
//
// Epilogue, codes: the reference dequantisation order
// fp32(fp32(acc) * fp32(sL[i] * sR[j])), then alpha and beta C; TF32:
// alpha acc + beta C.  Several K chunks: each CTA writes its partial sums
// and a reduction kernel adds them in a fixed order before the epilogue.
//
// Warp roles per CTA (192 threads): warp 0 issues TMA loads of 128 x 128-byte
// and BN x 128-byte K tiles (128-byte swizzle) into a ring of shared-memory
// stages; one thread of warp 1 issues the MMAs (M = 128, N = BN <= 256, 32
// bytes of K per instruction); warps 2..5 read the accumulator back with
// tcgen05.ld (TMEM lane = output row) and run the epilogue.  All waits are
// bounded; on expiry the kernel latches LRAMM_ERR_TIMEOUT, drains its own
// copies and MMAs, frees TMEM and returns.
#include "tc_common.cuh"

namespace lramm {
namespace {

using namespace tc;

constexpr int kQM = 128;         // output rows per CTA = TMEM lanes
constexpr int kQKB = 128;        // K bytes per stage: one 128-byte swizzle row
constexpr int kQThreads = 192;
constexpr int kQMaxStages = 8;
constexpr int kQChunkBlocks = 16;  // BF16 codes: 16 x 64 = 1024 products per exact FP32 partial

enum { kKindBF16 = 0, kKindFP8 = 1, kKindTF32 = 2 };

__host__ __device__ constexpr int kind_elem_bytes(int kind) { return kind == kKindBF16 ? 2 : (kind == kKindFP8 ? 1 : 4); }

struct QtcParams {
  int64_t M, N;
  int kblocks, kb_per_chunk, chunks;
  int bn, stages;
  uint32_t a_bytes, b_bytes, tmem_cols;
  int per_row;
  const float* sL;
  const float* sR;
  float alpha, beta;
  const float* C;
  int64_t ldc;
  float* D;
  int64_t ldd;
  float* part;   // chunks > 1: chunks x M x N partial sums
  int scaled;    // codes: dequantise with sL, sR; TF32: no scales
  int tma_store; // one chunk, beta = 0, D a valid TMA target: 32 x 32 blocks stored by TMA
  int nstg;      // staging blocks per epilogue warp (stores in flight per warp)
  int* status;
};

// Instruction descriptor: D F32 (bits 4-5 = 1); A and B formats at bits
// 7-9 and 10-12 (kind::f16: BF16 = 1; kind::f8f6f4: E4M3 = 0; kind::tf32:
// TF32 = 2); both K-major (bits 15, 16 = 0); N >> 3 at bit 17, M >> 4 at
// bit 24.
template <int KIND>
__device__ __forceinline__ uint32_t idesc_kind(int M, int N) {
  const uint32_t fmt = KIND == kKindBF16 ? 1u : (KIND == kKindFP8 ? 0u : 2u);
  return (1u << 4) | (fmt << 7) | (fmt << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void mma_kind(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  if (KIND == kKindBF16)
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  else if (KIND == kKindFP8)
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
__device__ __forceinline__ void epi_bar8() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

template <int KIND>
__global__ void __launch_bounds__(kQThreads, 2)
qgemm_tc_kernel(const __grid_constant__ CUtensorMap tmL, const __grid_constant__ CUtensorMap tmR,
                const __grid_constant__ CUtensorMap tmD, QtcParams p) {
  constexpr int kStageK = kQKB / kind_elem_bytes(KIND);   // K elements per stage
  extern __shared__ uint8_t q_smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(q_smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + static_cast<size_t>(p.stages) * p.a_bytes;
  __shared__ __align__(8) uint64_t full_bar[kQMaxStages], empty_bar[kQMaxStages], tmem_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  __shared__ float sR_sh[256];
  volatile int* abort_flag = &abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n0 = static_cast<int64_t>(blockIdx.x) * p.bn;
  const int64_t m0 = static_cast<int64_t>(blockIdx.y) * kQM;
  const int chunk = blockIdx.z;
  const int kb0 = chunk * p.kb_per_chunk;
  const int kb1 = min(p.kblocks, kb0 + p.kb_per_chunk);
  const int nkb = kb1 - kb0;

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
      const int k0 = (kb0 + i) * kStageK;
      tma_load_2d(sA + static_cast<size_t>(s) * p.a_bytes, &tmL, &full_bar[s], k0, static_cast<int>(m0));
      tma_load_2d(sB + static_cast<size_t>(s) * p.b_bytes, &tmR, &full_bar[s], k0, static_cast<int>(n0));
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
    const uint32_t idesc = idesc_kind<KIND>(kQM, p.bn);
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
      for (int kk = 0; kk < kQKB / 32; ++kk)  // 32 bytes of K per instruction
        mma_kind<KIND>(tmem, kmajor_sw128_desc(a_base + kk * 32), kmajor_sw128_desc(b_base + kk * 32), idesc,
                       (i > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&empty_bar[s]);
    }
    mma_commit(&tmem_bar);
  } else if (warp >= 2) {
    // ---- epilogue: TMEM lanes 32q .. 32q+31 are rows m0 + 32q + lane
    const int q = warp & 3;
    const int et = threadIdx.x - 64;   // 0 .. 127
    if (p.chunks == 1) {
      for (int j = et; j < p.bn; j += 128) {
        const int64_t col = n0 + j;
        sR_sh[j] = col < p.N ? (!p.scaled ? 1.f : (p.per_row ? p.sR[col] : p.sR[0])) : 0.f;
      }
    }
    epi_bar();
    volatile int zero = 0;  // wait for the MMAs even after an abort: they read shared memory
    const bool ok = mbar_wait(&tmem_bar, 0, &zero);
    tc_fence_after();
    const int64_t rbase = m0 + q * 32;
    const float sl_own = (p.chunks == 1 && rbase + lane < p.M)
                             ? (!p.scaled ? 1.f : (p.per_row ? p.sL[rbase + lane] : p.sL[0]))
                             : 0.f;
    if (p.tma_store) {
      // Each lane owns one output row of the block: the dequantised values go
      // to a staging block in the 128-byte swizzled layout (16-byte chunk c
      // of row r at chunk position c ^ (r mod 8)) and one lane stores the
      // block with a TMA bulk copy; nstg staging blocks per warp rotate, so
      // that many stores of a warp are in flight (the output write is what
      // bounds this product).  The blocks live in the operand ring, free once
      // the accumulator is complete: every copy into the ring was consumed by
      // an MMA before tmem_bar arrived.
      // The TMEM load of the next 32 columns is in flight while this block
      // is scaled, staged and stored.
      const uint32_t trow = tmem + (static_cast<uint32_t>(q * 32) << 16);
      uint32_t v[32], vn[32];
      tmem_ld32_issue(trow, v);
      tmem_ld_wait(v);
      for (int c0 = 0, nb = 0; c0 < p.bn; c0 += 32, ++nb) {
        const bool more = c0 + 32 < p.bn;
        if (more) tmem_ld32_issue(trow + static_cast<uint32_t>(c0 + 32), vn);
        float* stg = reinterpret_cast<float*>(sA) + (q * p.nstg + nb % p.nstg) * 1024;
        if (nb >= p.nstg) {   // this staging block's previous store has finished reading it
          if (lane == 0) {
            if (p.nstg == 4) asm volatile("cp.async.bulk.wait_group.read 3;" ::: "memory");
            else asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
          }
          __syncwarp();
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          float o[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float sr = sR_sh[c0 + 4 * c + e];
            const float x = __uint_as_float(v[4 * c + e]);
            o[e] = p.scaled ? __fmul_rn(p.alpha, __fmul_rn(x, __fmul_rn(sl_own, sr))) : __fmul_rn(p.alpha, x);
          }
          *reinterpret_cast<float4*>(stg + lane * 32 + ((c ^ (lane & 7)) << 2)) = make_float4(o[0], o[1], o[2], o[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0 && ok && rbase < p.M && n0 + c0 < p.N) {   // TMA clips the block at M and N
          asm volatile(
              "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                  reinterpret_cast<uint64_t>(&tmD)),
              "r"(static_cast<int>(n0 + c0)), "r"(static_cast<int>(rbase)), "r"(smem_u32(stg))
              : "memory");
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
        if (more) {
          tmem_ld_wait(vn);
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = vn[j];
        }
      }
      // the staging blocks must be read out before the CTA exits; the global
      // writes complete by themselves (visible at kernel completion)
      if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      __syncwarp();
    } else {
      // Each 32 x 32 block (rows = this warp's TMEM lanes) is transposed
      // through shared memory so that a store instruction writes 32
      // consecutive columns of one row (128 bytes); the 32 x 33 blocks live
      // in the operand ring, free once the accumulator is complete.
      float* T = reinterpret_cast<float*>(sA) + q * (32 * 33);
      for (int c0 = 0; c0 < p.bn; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(c0), v);
        __syncwarp();
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) T[lane * 33 + jj] = v[jj];
        __syncwarp();
        const int64_t col = n0 + c0 + lane;
        const bool col_ok = ok && col < p.N;
        const float sr = p.chunks == 1 ? sR_sh[c0 + lane] : 0.f;
#pragma unroll 4
        for (int r = 0; r < 32; ++r) {
          const float x = T[r * 33 + lane];
          const float sl = __shfl_sync(0xffffffffu, sl_own, r);
          const int64_t row = rbase + r;
          if (!col_ok || row >= p.M) continue;
          if (p.chunks > 1) {
            p.part[(static_cast<int64_t>(chunk) * p.M + row) * p.N + col] = x;
          } else {
            float o = p.scaled ? __fmul_rn(p.alpha, __fmul_rn(x, __fmul_rn(sl, sr))) : __fmul_rn(p.alpha, x);
            if (p.beta != 0.f) o = fmaf(p.beta, p.C[row * p.ldc + col], o);
            p.D[row * p.ldd + col] = o;
          }
        }
        __syncwarp();
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

// Persistent form of qgemm_tc_kernel for one K chunk with the output stored
// by TMA and no beta C term (the E3 shape: thousands of 128 x 256 tiles of
// a short-K product, bound by writing its FP32 output).  One CTA per SM
// walks the tiles t = blockIdx.x, + gridDim.x, ...: the operand ring keeps
// loading across tiles, and two 256-column TMEM accumulators let the MMAs of
// the next tile run while the epilogue warps drain the current one, so the
// output stream does not pause between tiles (with independent CTAs it
// stopped whenever both CTAs of an SM were loading or multiplying).  The
// arithmetic and the stores are those of qgemm_tc_kernel's TMA-store
// epilogue, so the results are bit-identical.
constexpr int kPStages = 2;       // operand ring (48 KB per stage at BN = 256)
constexpr int kPStg = 4;          // staging blocks of 4 KB per epilogue warp
constexpr int kPThreads = 320;    // warp 0 TMA, warp 1 MMA, warps 2..9 epilogue (two per TMEM lane quadrant)
constexpr int kPBN = 256;         // tile width (the launcher requires BN = 256)

template <int KIND, bool A1>   // A1: alpha == 1 (the multiply by alpha is exact and skipped)
__global__ void __launch_bounds__(kPThreads, 1)
qgemm_tcp_kernel(const __grid_constant__ CUtensorMap tmL, const __grid_constant__ CUtensorMap tmR,
                 const __grid_constant__ CUtensorMap tmD, QtcParams p, int ntn, int64_t ntiles) {
  constexpr int kStageK = kQKB / kind_elem_bytes(KIND);
  extern __shared__ uint8_t q_smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(q_smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + static_cast<size_t>(kPStages) * p.a_bytes;
  float* stg_base = reinterpret_cast<float*>(sB + static_cast<size_t>(kPStages) * p.b_bytes);   // 8 x kPStg x 4 KB
  float* sR_sh = stg_base + 8 * kPStg * 1024;                                                    // p.bn floats
  __shared__ __align__(8) uint64_t full_bar[kPStages], empty_bar[kPStages], accf[2], acce[2], done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  volatile int* abort_flag = &abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = p.kblocks;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kPStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&accf[a], 1);
      mbar_init(&acce[a], 8);   // one arrival per epilogue warp
    }
    mbar_init(&done_bar, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: every K block of every tile of this CTA, in order
    int64_t it = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const int m0 = static_cast<int>(t / ntn) * kQM, n0 = static_cast<int>(t % ntn) * p.bn;
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const int s = static_cast<int>(it % kPStages);
        if (it >= kPStages && !mbar_wait(&empty_bar[s], static_cast<uint32_t>((it / kPStages) & 1) ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        mbar_expect_tx(&full_bar[s], p.a_bytes + p.b_bytes);
        tma_load_2d(sA + static_cast<size_t>(s) * p.a_bytes, &tmL, &full_bar[s], kb * kStageK, m0);
        tma_load_2d(sB + static_cast<size_t>(s) * p.b_bytes, &tmR, &full_bar[s], kb * kStageK, n0);
      }
    }
    if (!ok) {
      set_status(p.status, LRAMM_ERR_TIMEOUT);
      abort_sh = 1;
      volatile int zero = 0;   // the copies still in flight land before the CTA exits
      for (int64_t i = it > kPStages ? it - kPStages : 0; i < it; ++i)
        mbar_wait(&full_bar[i % kPStages], static_cast<uint32_t>((i / kPStages) & 1), &zero);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: accumulator j & 1 for the j-th tile of this CTA
    const uint32_t idesc = idesc_kind<KIND>(kQM, p.bn);
    int64_t it = 0;
    bool ok = true;
    int j = 0;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++j) {
      const int a = j & 1;
      if (j >= 2 && !mbar_wait(&acce[a], static_cast<uint32_t>((j / 2 - 1) & 1), abort_flag)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d = tmem + static_cast<uint32_t>(a * 256);
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const int s = static_cast<int>(it % kPStages);
        if (!mbar_wait(&full_bar[s], static_cast<uint32_t>((it / kPStages) & 1), abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a_base = smem_u32(sA + static_cast<size_t>(s) * p.a_bytes);
        const uint32_t b_base = smem_u32(sB + static_cast<size_t>(s) * p.b_bytes);
#pragma unroll
        for (int kk = 0; kk < kQKB / 32; ++kk)  // 32 bytes of K per instruction
          mma_kind<KIND>(d, kmajor_sw128_desc(a_base + kk * 32), kmajor_sw128_desc(b_base + kk * 32), idesc,
                         (kb > 0 || kk > 0) ? 1u : 0u);
        mma_commit(&empty_bar[s]);
      }
      if (ok) mma_commit(&accf[a]);
    }
    if (!ok) {
      set_status(p.status, LRAMM_ERR_TIMEOUT);
      abort_sh = 1;
    }
    // every MMA issued has finished before the CTA frees TMEM and exits
    mma_commit(&done_bar);
    volatile int zero = 0;
    mbar_wait(&done_bar, 0, &zero);
  } else if (warp >= 2) {
    // ---- epilogue: TMEM lanes 32q .. 32q+31 are rows m0 + 32q + lane;
    // warps 2..5 take the tile's first half of the columns, 6..9 the second
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    const int et = threadIdx.x - 64;   // 0 .. 255
    float* stg0 = stg_base + (warp - 2) * kPStg * 1024;
    const int cbeg = half * (kPBN / 2);
    int sc = 0;   // staging blocks used by this warp
    bool ok = true;
    int j = 0;
    // the scales of a tile are loaded one tile ahead (their latency was the
    // epilogue's main stall): thread et holds column et's scale, each lane
    // its row's
    auto col_scale = [&](int64_t tt) {
      const int64_t col = (tt % ntn) * kPBN + et;
      return tt < ntiles && col < p.N ? (p.per_row ? p.sR[col] : p.sR[0]) : 0.f;
    };
    auto row_scale = [&](int64_t tt) {
      const int64_t row = (tt / ntn) * kQM + q * 32 + lane;
      return tt < ntiles && row < p.M ? (p.per_row ? p.sL[row] : p.sL[0]) : 0.f;
    };
    float sr_next = col_scale(blockIdx.x), sl_next = row_scale(blockIdx.x);
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
      const int a = j & 1;
      const int64_t m0 = (t / ntn) * kQM, n0 = (t % ntn) * p.bn;
      epi_bar8();   // every epilogue warp is done with the previous tile's column scales
      sR_sh[et] = sr_next;
      const float sl_own = sl_next;
      sr_next = col_scale(t + gridDim.x);
      sl_next = row_scale(t + gridDim.x);
      epi_bar8();
      const int64_t rbase = m0 + q * 32;
      // after an abort the warp keeps walking the tiles through the two
      // named barriers above (so no epilogue warp waits on one that left)
      // and does nothing else
      if (ok && !mbar_wait(&accf[a], static_cast<uint32_t>((j / 2) & 1), abort_flag)) ok = false;
      if (!ok) continue;
      tc_fence_after();
      const uint32_t trow = tmem + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(a * 256);
      // one 32 x 32 block: scale, stage (128-byte swizzle), store by TMA
      auto emit = [&](const uint32_t(&v)[32], int c0) {
        float* stg = stg0 + (sc % kPStg) * 1024;
        if (sc >= kPStg) {   // this staging block's previous store has been read out
          if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 3;" ::: "memory");
          __syncwarp();
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float4 sr = *reinterpret_cast<const float4*>(sR_sh + c0 + 4 * c);
          float o[4] = {__fmul_rn(__uint_as_float(v[4 * c]), __fmul_rn(sl_own, sr.x)),
                        __fmul_rn(__uint_as_float(v[4 * c + 1]), __fmul_rn(sl_own, sr.y)),
                        __fmul_rn(__uint_as_float(v[4 * c + 2]), __fmul_rn(sl_own, sr.z)),
                        __fmul_rn(__uint_as_float(v[4 * c + 3]), __fmul_rn(sl_own, sr.w))};
          if (!A1)
#pragma unroll
            for (int e = 0; e < 4; ++e) o[e] = __fmul_rn(p.alpha, o[e]);
          *reinterpret_cast<float4*>(stg + lane * 32 + ((c ^ (lane & 7)) << 2)) = make_float4(o[0], o[1], o[2], o[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0 && rbase < p.M && n0 + c0 < p.N) {   // TMA clips the block at M and N
          asm volatile(
              "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                  reinterpret_cast<uint64_t>(&tmD)),
              "r"(static_cast<int>(n0 + c0)), "r"(static_cast<int>(rbase)), "r"(smem_u32(stg))
              : "memory");
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
        ++sc;
      };
      // the warp's four blocks, each TMEM load in flight while the previous
      // block is emitted (two register sets, no copies)
      uint32_t va[32], vb[32];
      tmem_ld32_issue(trow + static_cast<uint32_t>(cbeg), va);
      tmem_ld_wait(va);
      tmem_ld32_issue(trow + static_cast<uint32_t>(cbeg + 32), vb);
      emit(va, cbeg);
      tmem_ld_wait(vb);
      tmem_ld32_issue(trow + static_cast<uint32_t>(cbeg + 64), va);
      emit(vb, cbeg + 32);
      tmem_ld_wait(va);
      tmem_ld32_issue(trow + static_cast<uint32_t>(cbeg + 96), vb);
      emit(va, cbeg + 64);
      tmem_ld_wait(vb);
      emit(vb, cbeg + 96);
      // accumulator a drained: the MMAs of tile j + 2 may overwrite it
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[a])) : "memory");
    }
    if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    __syncwarp();
    if (!ok) {
      set_status(p.status, LRAMM_ERR_TIMEOUT);
      abort_sh = 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// D = dequantised sum over chunks: tot = sum_c part[c] in a fixed order (as
// 32-bit integers for BF16 codes, whose total may pass 2^24; in FP32
// otherwise), then fp32(fp32(tot) * fp32(sL * sR)) (or tot unscaled), alpha
// and beta C.
template <bool INT_SUM>
__global__ void qgemm_tc_reduce_kernel(QtcParams p) {
  const int64_t total = p.M * p.N;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / p.N, j = e - i * p.N;
    float totf;
    if (INT_SUM) {
      int tot = 0;
      for (int c = 0; c < p.chunks; ++c) tot += __float2int_rn(p.part[static_cast<int64_t>(c) * total + e]);
      totf = static_cast<float>(tot);
    } else {
      totf = 0.f;
      for (int c = 0; c < p.chunks; ++c) totf += p.part[static_cast<int64_t>(c) * total + e];
    }
    float o;
    if (p.scaled) {
      const float sp = __fmul_rn(p.per_row ? p.sL[i] : p.sL[0], p.per_row ? p.sR[j] : p.sR[0]);
      o = __fmul_rn(p.alpha, __fmul_rn(totf, sp));
    } else {
      o = __fmul_rn(p.alpha, totf);
    }
    if (p.beta != 0.f) o = fmaf(p.beta, p.C[i * p.ldc + j], o);
    p.D[i * p.ldd + j] = o;
  }
}

// ---------------------------------------------------------------------------
// A sum of QM terms in one pass over the output (the lead / tail E3 of
// Algorithm 3 with split-precision residuals):
//   D = alpha sum_t fp32(fp32(acc_t) * fp32(sL_t[i] sR_t[j])) + beta C,
//   acc_t[i][j] = sum_k L_t[i][k] R_t[j][k]    (BF16 operands, K-major)
// Term t accumulates in its own TMEM region (columns t * BN ..); the K blocks
// of all terms stream through one ring.  Scaled terms hold INT8 codes (exact
// sums of at most 1024 products); an unscaled term holds exact BF16 values
// (the MXFP4 tail: e2m1 code times its block's power of two) whose products
// the tensor core sums in FP32.  The epilogue adds the terms in order, each
// rounded as a separate pass would round it:
//   o = fp32(alpha T_0) (+ beta C), then o = fp32(o + fp32(alpha T_t)).
constexpr int kMaxTerms = 4;
constexpr int kTermBN = 64;   // output columns per CTA: 4 regions of 64 TMEM columns, two CTAs per SM

struct QtermsParams {
  int64_t M, N;
  int nterms, kb_total;
  int kb_start[kMaxTerms + 1];   // first ring block of each term; kb_start[nterms] = kb_total
  const float* sL[kMaxTerms];    // nullptr: unscaled term
  const float* sR[kMaxTerms];
  int per_row;
  int stages;
  uint32_t a_bytes, b_bytes, tmem_cols;
  float alpha, beta;
  const float* C;
  int64_t ldc;
  float* D;
  int64_t ldd;
  int tma_store;
  int* status;
};

__global__ void __launch_bounds__(kQThreads, 2)
qterms_tc_kernel(const __grid_constant__ CUtensorMap tmL0, const __grid_constant__ CUtensorMap tmL1,
                 const __grid_constant__ CUtensorMap tmL2, const __grid_constant__ CUtensorMap tmL3,
                 const __grid_constant__ CUtensorMap tmR0, const __grid_constant__ CUtensorMap tmR1,
                 const __grid_constant__ CUtensorMap tmR2, const __grid_constant__ CUtensorMap tmR3,
                 const __grid_constant__ CUtensorMap tmD, QtermsParams p) {
  constexpr int kStageK = kQKB / 2;   // 64 BF16 per stage
  extern __shared__ uint8_t qt_smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(qt_smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + static_cast<size_t>(p.stages) * p.a_bytes;
  __shared__ __align__(8) uint64_t full_bar[kQMaxStages], empty_bar[kQMaxStages], tmem_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  __shared__ float sR_sh[kMaxTerms][kTermBN];
  volatile int* abort_flag = &abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n0 = static_cast<int64_t>(blockIdx.x) * kTermBN;
  const int64_t m0 = static_cast<int64_t>(blockIdx.y) * kQM;
  const int nkb = p.kb_total;

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
    // ---- TMA producer: the terms' K blocks in order.  Each term's loads
    // name their own tensor-map parameters directly (no map is picked
    // through a runtime index).
    int issued = 0;
    bool ok = true;
    auto load_term = [&](const CUtensorMap* ml, const CUtensorMap* mr, int t) {
      for (int i = p.kb_start[t]; ok && i < p.kb_start[t + 1]; ++i) {
        const int s = i % p.stages;
        if (i >= p.stages && !mbar_wait(&empty_bar[s], ((i / p.stages) & 1) ^ 1, abort_flag)) {
          ok = false;
          break;
        }
        mbar_expect_tx(&full_bar[s], tx_bytes);
        const int k0 = (i - p.kb_start[t]) * kStageK;
        tma_load_2d(sA + static_cast<size_t>(s) * p.a_bytes, ml, &full_bar[s], k0, static_cast<int>(m0));
        tma_load_2d(sB + static_cast<size_t>(s) * p.b_bytes, mr, &full_bar[s], k0, static_cast<int>(n0));
        ++issued;
      }
    };
    load_term(&tmL0, &tmR0, 0);
    if (p.nterms > 1) load_term(&tmL1, &tmR1, 1);
    if (p.nterms > 2) load_term(&tmL2, &tmR2, 2);
    if (p.nterms > 3) load_term(&tmL3, &tmR3, 3);
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
    // ---- MMA issuer: term t into TMEM columns t * BN ..
    const uint32_t idesc = idesc_kind<kKindBF16>(kQM, kTermBN);
    int t = 0;
    for (int i = 0; i < nkb; ++i) {
      while (i >= p.kb_start[t + 1]) ++t;
      const int s = i % p.stages;
      if (!mbar_wait(&full_bar[s], (i / p.stages) & 1, abort_flag)) {
        set_status(p.status, LRAMM_ERR_TIMEOUT);
        abort_sh = 1;
        break;
      }
      tc_fence_after();
      const uint32_t a_base = smem_u32(sA + static_cast<size_t>(s) * p.a_bytes);
      const uint32_t b_base = smem_u32(sB + static_cast<size_t>(s) * p.b_bytes);
      const uint32_t d = tmem + static_cast<uint32_t>(t * kTermBN);
      const bool first = i == p.kb_start[t];
#pragma unroll
      for (int kk = 0; kk < kQKB / 32; ++kk)  // 16 BF16 (32 bytes) of K per instruction
        mma_kind<kKindBF16>(d, kmajor_sw128_desc(a_base + kk * 32), kmajor_sw128_desc(b_base + kk * 32), idesc,
                            (!first || kk > 0) ? 1u : 0u);
      mma_commit(&empty_bar[s]);
    }
    mma_commit(&tmem_bar);
  } else if (warp >= 2) {
    // ---- epilogue: TMEM lanes 32q .. 32q+31 are rows m0 + 32q + lane
    const int q = warp & 3;
    const int et = threadIdx.x - 64;   // 0 .. 127
    for (int e = et; e < p.nterms * kTermBN; e += 128) {
      const int t = e / kTermBN, j = e - t * kTermBN;
      const int64_t col = n0 + j;
      sR_sh[t][j] = col < p.N ? (p.sR[t] ? (p.per_row ? p.sR[t][col] : p.sR[t][0]) : 1.f) : 0.f;
    }
    epi_bar();
    volatile int zero = 0;  // wait for the MMAs even after an abort: they read shared memory
    const bool ok = mbar_wait(&tmem_bar, 0, &zero);
    tc_fence_after();
    const int64_t rbase = m0 + q * 32;
    const int64_t row_own = rbase + lane;
    float sl_own[kMaxTerms];
#pragma unroll
    for (int t = 0; t < kMaxTerms; ++t)
      sl_own[t] = (t < p.nterms && row_own < p.M)
                      ? (p.sL[t] ? (p.per_row ? p.sL[t][row_own] : p.sL[t][0]) : 1.f)
                      : 0.f;
    // TMEM blocks (column block, term) in order, each load in flight while
    // the previous block is combined (and, after a column block's last
    // term, while that block is staged and stored)
    const uint32_t trow = tmem + (static_cast<uint32_t>(q * 32) << 16);
    uint32_t vn[32];
    tmem_ld32_issue(trow, vn);
    for (int c0 = 0, nb = 0; c0 < kTermBN; c0 += 32, ++nb) {
      // this lane's row, columns c0 .. c0+31: the terms combined in order
      float o[32];
      for (int t = 0; t < p.nterms; ++t) {
        uint32_t v[32];
        tmem_ld_wait(vn);
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = vn[j];
        if (t + 1 < p.nterms)
          tmem_ld32_issue(trow + static_cast<uint32_t>((t + 1) * kTermBN + c0), vn);
        else if (c0 + 32 < kTermBN)
          tmem_ld32_issue(trow + static_cast<uint32_t>(c0 + 32), vn);
        const bool scaled = p.sL[t] != nullptr;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float x = __uint_as_float(v[j]);
          const float term = scaled ? __fmul_rn(p.alpha, __fmul_rn(x, __fmul_rn(sl_own[t], sR_sh[t][c0 + j])))
                                    : __fmul_rn(p.alpha, x);
          o[j] = t == 0 ? term : __fadd_rn(o[j], term);
        }
        if (t == 0 && p.beta != 0.f && row_own < p.M) {   // beta C joins the first term
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int64_t col = n0 + c0 + j;
            if (col < p.N) o[j] = fmaf(p.beta, p.C[row_own * p.ldc + col], o[j]);
          }
        }
      }
      if (p.tma_store) {
        // swizzled 32 x 32 staging block in the (now idle) operand ring, stored by TMA
        float* stg = reinterpret_cast<float*>(sA) + (q * 2 + (nb & 1)) * 1024;
        if (nb >= 2) {
          if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
          __syncwarp();
        }
#pragma unroll
        for (int c = 0; c < 8; ++c)
          *reinterpret_cast<float4*>(stg + lane * 32 + ((c ^ (lane & 7)) << 2)) =
              make_float4(o[4 * c], o[4 * c + 1], o[4 * c + 2], o[4 * c + 3]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0 && ok && rbase < p.M && n0 + c0 < p.N) {   // TMA clips the block at M and N
          asm volatile(
              "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                  reinterpret_cast<uint64_t>(&tmD)),
              "r"(static_cast<int>(n0 + c0)), "r"(static_cast<int>(rbase)), "r"(smem_u32(stg))
              : "memory");
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
      } else {
        // 32 x 32 block transposed through shared memory: each store writes
        // 32 consecutive columns of one row
        float* T = reinterpret_cast<float*>(sA) + q * (32 * 33);
        __syncwarp();
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) T[lane * 33 + jj] = o[jj];
        __syncwarp();
        const int64_t col = n0 + c0 + lane;
        const bool col_ok = ok && col < p.N;
#pragma unroll 4
        for (int r = 0; r < 32; ++r) {
          const int64_t row = rbase + r;
          if (!col_ok || row >= p.M) continue;
          p.D[row * p.ldd + col] = T[r * 33 + lane];
        }
        __syncwarp();
      }
    }
    if (p.tma_store) {   // staging blocks read out before the CTA exits
      if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      __syncwarp();
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

constexpr int kQSmemBudget = 232448 - 4096;  // opt-in maximum minus alignment slack and static shared memory

struct QtcShape {
  int kblocks, kb_per_chunk, chunks, bn, stages;
  int64_t mtiles, ntiles;
};

QtcShape qtc_shape(int kind, int64_t M, int64_t N, int64_t K) {
  QtcShape sh{};
  const int stage_k = kQKB / kind_elem_bytes(kind);
  sh.kblocks = static_cast<int>(ceil_div(K, stage_k));
  sh.bn = static_cast<int>(N >= 256 ? 256 : round_up(N, 16));
  // short K and a wide output (E3: m x n, K = r; the rank-l updates of the
  // range-finder backward): a 2-stage ring so that two CTAs share an SM and
  // one CTA's epilogue (the HBM-bound part) overlaps the other's loads and MMAs
  const bool wide = N >= 1024 && K * kind_elem_bytes(kind) <= 2048;
  sh.mtiles = ceil_div(M, kQM);
  sh.ntiles = ceil_div(N, sh.bn);
  const int64_t tiles = sh.mtiles * sh.ntiles;
  // chunk limit: exactness for BF16 codes, none otherwise
  const int cap = kind == kKindBF16 ? kQChunkBlocks : sh.kblocks;
  int kpc = cap;
  if (tiles < 64) {  // few output tiles: split K further for parallelism (at least 4 blocks per CTA)
    const int64_t want = ceil_div(static_cast<int64_t>(sh.kblocks) * tiles, 128);
    kpc = static_cast<int>(want < 4 ? 4 : (want > cap ? cap : want));
  }
  if (kpc > sh.kblocks) kpc = sh.kblocks;
  if (kpc < 1) kpc = 1;
  sh.kb_per_chunk = kpc;
  sh.chunks = static_cast<int>(ceil_div(sh.kblocks, kpc));
  const int stage_bytes = (kQM + sh.bn) * kQKB;
  int st = (kQSmemBudget - 1024) / stage_bytes;
  if (st > kQMaxStages) st = kQMaxStages;
  if (st > sh.kb_per_chunk) st = sh.kb_per_chunk;
  if (st < 2) st = 2;
  // a 2-stage ring (48 KB per stage at BN = 256) leaves room for two CTAs per SM
  if (wide || (sh.kb_per_chunk <= 8 && sh.bn <= 128)) st = 2;
  sh.stages = st;
  return sh;
}

int prec_kind(int prec) { return prec == LRAMM_P_INT8 ? kKindBF16 : kKindFP8; }

bool tc_operands_ok(int kind, const void* L, const void* R, int64_t ldl, int64_t ldr, int64_t M, int64_t N,
                    int64_t K) {
  if (M <= 0 || N <= 0 || K <= 0 || M > INT32_MAX || N > INT32_MAX || K > INT32_MAX) return false;
  const int eb = kind_elem_bytes(kind);
  // TMA: 16-byte aligned bases and row pitches
  return (reinterpret_cast<uintptr_t>(L) % 16) == 0 && (reinterpret_cast<uintptr_t>(R) % 16) == 0 &&
         (ldl * eb) % 16 == 0 && (ldr * eb) % 16 == 0 && ldl >= K && ldr >= K;
}

lramm_status launch_tc(int kind, const void* L, const void* R, int64_t M, int64_t N, int64_t K, int64_t ldl,
                       int64_t ldr, QtcParams p, cudaStream_t s) {
  const QtcShape sh = qtc_shape(kind, M, N, K);
  if (sh.chunks > 1 && (!p.part)) return LRAMM_ERR_WORKSPACE;
  if (sh.mtiles > 65535 || sh.chunks > 65535) return LRAMM_ERR_UNSUPPORTED;
  p.M = M;
  p.N = N;
  p.kblocks = sh.kblocks;
  p.kb_per_chunk = sh.kb_per_chunk;
  p.chunks = sh.chunks;
  p.bn = sh.bn;
  p.a_bytes = kQM * kQKB;
  p.b_bytes = static_cast<uint32_t>(sh.bn) * kQKB;
  p.stages = sh.stages;
  uint32_t tc = 32;
  while (tc < static_cast<uint32_t>(sh.bn)) tc <<= 1;
  p.tmem_cols = tc;
  const int eb = kind_elem_bytes(kind);
  const CUtensorMapDataType dt = kind == kKindBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                 : kind == kKindFP8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                                    : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const uint32_t box_k = static_cast<uint32_t>(kQKB / eb);
  CUtensorMap mL, mR;
  if (!make_map_2d(&mL, dt, L, K, M, ldl * eb, box_k, kQM, CU_TENSOR_MAP_SWIZZLE_128B)) return LRAMM_ERR_CUDA;
  if (!make_map_2d(&mR, dt, R, K, N, ldr * eb, box_k, static_cast<uint32_t>(sh.bn), CU_TENSOR_MAP_SWIZZLE_128B))
    return LRAMM_ERR_CUDA;
  // TMA stores of the output: one K chunk, no beta C term, D 16-byte aligned
  // with a row pitch that is a multiple of 16 bytes
  CUtensorMap mD;
  // staging blocks of 4 KB in the operand ring: four per epilogue warp where
  // the ring holds 16, else two
  const uint32_t ring = static_cast<uint32_t>(p.stages) * (p.a_bytes + p.b_bytes);
  p.nstg = ring >= 16 * 4096 ? 4 : 2;
  p.tma_store = sh.chunks == 1 && p.beta == 0.f && ring >= 8 * 4096 &&
                (reinterpret_cast<uintptr_t>(p.D) % 16) == 0 &&
                (p.ldd * 4) % 16 == 0 && p.ldd >= N &&
                make_map_2d(&mD, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, p.D, N, M, p.ldd * 4, 32, 32,
                            CU_TENSOR_MAP_SWIZZLE_128B);
  if (!p.tma_store) mD = mL;   // unused
  // many output tiles of a one-chunk code product stored by TMA: the
  // persistent kernel, one CTA per SM
  const int64_t ntl = sh.mtiles * sh.ntiles;
  if (p.tma_store && p.scaled && sh.chunks == 1 && kind != kKindTF32 && sh.bn == 256 && ntl >= 4 * num_sms()) {
    const size_t psmem = 1024 + static_cast<size_t>(kPStages) * (p.a_bytes + p.b_bytes) +
                         static_cast<size_t>(8 * kPStg) * 4096 + sizeof(float) * p.bn;
    const unsigned gp = static_cast<unsigned>(num_sms());
    const int nt = static_cast<int>(sh.ntiles);
    const bool a1 = p.alpha == 1.f;
#define LRAMM_TCP(K, A)                                                                                      \
  do {                                                                                                       \
    LRAMM_CUDA_TRY(smem_cap(qgemm_tcp_kernel<K, A>, \
                                        (int)psmem));                                                        \
    qgemm_tcp_kernel<K, A><<<gp, kPThreads, psmem, s>>>(mL, mR, mD, p, nt, ntl);                              \
  } while (0)
    if (kind == kKindBF16) {
      if (a1) LRAMM_TCP(kKindBF16, true);
      else LRAMM_TCP(kKindBF16, false);
    } else {
      if (a1) LRAMM_TCP(kKindFP8, true);
      else LRAMM_TCP(kKindFP8, false);
    }
#undef LRAMM_TCP
    return last_launch();
  }
  const size_t smem = 1024 + static_cast<size_t>(p.stages) * (p.a_bytes + p.b_bytes);
  const dim3 grid(static_cast<unsigned>(sh.ntiles), static_cast<unsigned>(sh.mtiles), static_cast<unsigned>(sh.chunks));
  switch (kind) {
    case kKindBF16:
      LRAMM_CUDA_TRY(smem_cap(qgemm_tc_kernel<kKindBF16>, (int)smem));
      qgemm_tc_kernel<kKindBF16><<<grid, kQThreads, smem, s>>>(mL, mR, mD, p);
      break;
    case kKindFP8:
      LRAMM_CUDA_TRY(smem_cap(qgemm_tc_kernel<kKindFP8>, (int)smem));
      qgemm_tc_kernel<kKindFP8><<<grid, kQThreads, smem, s>>>(mL, mR, mD, p);
      break;
    default:
      LRAMM_CUDA_TRY(smem_cap(qgemm_tc_kernel<kKindTF32>, (int)smem));
      qgemm_tc_kernel<kKindTF32><<<grid, kQThreads, smem, s>>>(mL, mR, mD, p);
      break;
  }
  LRAMM_TRY(last_launch());
  if (sh.chunks > 1) {
    int64_t g = ceil_div(M * N, 256);
    if (g > num_sms() * 8) g = num_sms() * 8;
    if (kind == kKindBF16)
      qgemm_tc_reduce_kernel<true><<<static_cast<unsigned>(g), 256, 0, s>>>(p);
    else
      qgemm_tc_reduce_kernel<false><<<static_cast<unsigned>(g), 256, 0, s>>>(p);
    LRAMM_TRY(last_launch());
  }
  return LRAMM_OK;
}

}  // namespace

bool qgemm_tc_supported(int prec, const void* L, const void* R, int64_t ldl, int64_t ldr, int64_t M, int64_t N,
                        int64_t K) {
  if (prec != LRAMM_P_INT8 && prec != LRAMM_P_INT4 && prec != LRAMM_P_E4M3) return false;
  if (prec == LRAMM_P_INT4 && K >= 342000) return false;   // exact FP32 sums of products <= 49
  return tc_operands_ok(prec_kind(prec), L, R, ldl, ldr, M, N, K);
}

size_t qgemm_tc_part_floats(int prec, int64_t M, int64_t N, int64_t K) {
  const QtcShape sh = qtc_shape(prec_kind(prec), M, N, K);
  return sh.chunks > 1 ? static_cast<size_t>(sh.chunks) * M * N : 0;
}

lramm_status qgemm_tc(int prec, const void* L, const void* R, int64_t M, int64_t N, int64_t K, int64_t ldl,
                      int64_t ldr, int per_row, const float* sL, const float* sR, float alpha, float beta,
                      const float* C, int64_t ldc, float* D, int64_t ldd, float* part, size_t part_floats,
                      int* status, cudaStream_t s) {
  if (!qgemm_tc_supported(prec, L, R, ldl, ldr, M, N, K)) return LRAMM_ERR_UNSUPPORTED;
  if (part_floats < qgemm_tc_part_floats(prec, M, N, K)) return LRAMM_ERR_WORKSPACE;
  QtcParams p{};
  p.per_row = per_row;
  p.sL = sL;
  p.sR = sR;
  p.alpha = alpha;
  p.beta = beta;
  p.C = C;
  p.ldc = ldc;
  p.D = D;
  p.ldd = ldd;
  p.part = part;
  p.scaled = 1;
  p.status = status;
  return launch_tc(prec_kind(prec), L, R, M, N, K, ldl, ldr, p, s);
}

bool tgemm_tc_supported(const float* A, const float* B, int64_t lda, int64_t ldb, int64_t M, int64_t N, int64_t K) {
  return tc_operands_ok(kKindTF32, A, B, lda, ldb, M, N, K);
}

size_t tgemm_tc_part_floats(int64_t M, int64_t N, int64_t K) {
  const QtcShape sh = qtc_shape(kKindTF32, M, N, K);
  return sh.chunks > 1 ? static_cast<size_t>(sh.chunks) * M * N : 0;
}

lramm_status tgemm_tc(int64_t M, int64_t N, int64_t K, float alpha, const float* A, int64_t lda, const float* B,
                      int64_t ldb, float beta, float* C, int64_t ldc, float* part, size_t part_floats, int* status,
                      cudaStream_t s) {
  if (!tgemm_tc_supported(A, B, lda, ldb, M, N, K)) return LRAMM_ERR_UNSUPPORTED;
  if (part_floats < tgemm_tc_part_floats(M, N, K)) return LRAMM_ERR_WORKSPACE;
  QtcParams p{};
  p.per_row = 0;
  p.alpha = alpha;
  p.beta = beta;
  p.C = C;
  p.ldc = ldc;
  p.D = C;
  p.ldd = ldc;
  p.part = part;
  p.scaled = 0;
  p.status = status;
  return launch_tc(kKindTF32, A, B, M, N, K, lda, ldb, p, s);
}

bool qterms_tc_supported(int nterms, const void* const* L, const void* const* R, const int64_t* K, const int64_t* ldl,
                         const int64_t* ldr, const float* const* sL, int64_t M, int64_t N) {
  if (nterms < 1 || nterms > kMaxTerms) return false;
  for (int t = 0; t < nterms; ++t) {
    if (!tc_operands_ok(kKindBF16, L[t], R[t], ldl[t], ldr[t], M, N, K[t])) return false;
    if (sL[t] && K[t] > kQChunkBlocks * (kQKB / 2)) return false;   // exact integer sums: at most 1024 products
  }
  return M / kQM < 65535;
}

lramm_status qterms_tc(int nterms, const void* const* L, const void* const* R, const int64_t* K, const int64_t* ldl,
                       const int64_t* ldr, const float* const* sL, const float* const* sR, int per_row, int64_t M,
                       int64_t N, float alpha, float beta, const float* C, int64_t ldc, float* D, int64_t ldd,
                       int* status, cudaStream_t s) {
  if (!qterms_tc_supported(nterms, L, R, K, ldl, ldr, sL, M, N)) return LRAMM_ERR_UNSUPPORTED;
  if (beta != 0.f && !C) return LRAMM_ERR_INVALID_ARG;
  QtermsParams p{};
  p.M = M;
  p.N = N;
  p.nterms = nterms;
  constexpr int kStageK = kQKB / 2;
  int kb = 0;
  for (int t = 0; t < nterms; ++t) {
    p.kb_start[t] = kb;
    kb += static_cast<int>(ceil_div(K[t], kStageK));
    p.sL[t] = sL[t];
    p.sR[t] = sL[t] ? sR[t] : nullptr;
  }
  p.kb_start[nterms] = kb;
  for (int t = nterms + 1; t <= kMaxTerms; ++t) p.kb_start[t] = kb;
  p.kb_total = kb;
  p.per_row = per_row;
  p.a_bytes = kQM * kQKB;
  p.b_bytes = kTermBN * kQKB;
  p.stages = 3;
  p.tmem_cols = static_cast<uint32_t>(kMaxTerms * kTermBN);   // 256: two CTAs per SM
  p.alpha = alpha;
  p.beta = beta;
  p.C = C;
  p.ldc = ldc;
  p.D = D;
  p.ldd = ldd;
  p.status = status;
  CUtensorMap mL[kMaxTerms], mR[kMaxTerms];
  for (int t = 0; t < kMaxTerms; ++t) {
    const int u = t < nterms ? t : 0;   // unused slots repeat term 0's maps
    if (!make_map_2d(&mL[t], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, L[u], K[u], M, ldl[u] * 2, kQKB / 2, kQM,
                     CU_TENSOR_MAP_SWIZZLE_128B) ||
        !make_map_2d(&mR[t], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, R[u], K[u], N, ldr[u] * 2, kQKB / 2, kTermBN,
                     CU_TENSOR_MAP_SWIZZLE_128B))
      return LRAMM_ERR_CUDA;
  }
  CUtensorMap mD;
  p.tma_store = beta == 0.f && (reinterpret_cast<uintptr_t>(D) % 16) == 0 && (ldd * 4) % 16 == 0 && ldd >= N &&
                make_map_2d(&mD, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, D, N, M, ldd * 4, 32, 32, CU_TENSOR_MAP_SWIZZLE_128B);
  if (!p.tma_store) mD = mL[0];   // unused
  const size_t smem = 1024 + static_cast<size_t>(p.stages) * (p.a_bytes + p.b_bytes);
  LRAMM_CUDA_TRY(smem_cap(qterms_tc_kernel, (int)smem));
  const dim3 grid(static_cast<unsigned>(ceil_div(N, kTermBN)), static_cast<unsigned>(ceil_div(M, kQM)));
  qterms_tc_kernel<<<grid, kQThreads, smem, s>>>(mL[0], mL[1], mL[2], mL[3], mR[0], mR[1], mR[2], mR[3], mD, p);
  return last_launch();
}

}  // namespace lramm
