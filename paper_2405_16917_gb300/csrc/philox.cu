// Philox4x32-10 and the Gaussian test matrix Omega of the randomized range
// finder (paper Sec. 2.2, "Gaussian sampling").
//
// Philox4x32-10 (Salmon et al., SC'11): 128-bit counter, 64-bit key; a round
// multiplies counter words 0 and 2 by 0xD2511F53 / 0xCD9E8D57, splits the
// 64-bit products and mixes them with words 1, 3 and the key; the key is
// bumped by 0x9E3779B9 / 0xBB67AE85 between the ten rounds.
// Counter of block n for stream s: (lo32 n, hi32 n, s, 0); key (lo32 seed,
// hi32 seed).  Box-Muller on the word pairs (0,1) and (2,3) with exact FP32
// uniforms u1 = ((x >> 8) + 1) 2^-24 and u2 = (2 (y >> 9) + 1) 2^-24.
#include "common.cuh"

namespace lramm {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

__device__ __forceinline__ uint4 philox_block(uint64_t seed, uint32_t sid, uint64_t n) {
  return philox4x32_10(make_uint4((uint32_t)n, (uint32_t)(n >> 32), sid, 0u), (uint32_t)seed,
                       (uint32_t)(seed >> 32));
}

// ln(u1) with relative accuracy over the whole range: for u1 >= 1/2 the
// logarithm is taken as log1p of the exact (negative) distance to 1.
__device__ __forceinline__ void box_muller(uint32_t x, uint32_t y, float& z0, float& z1) {
  const uint32_t t = x >> 8;  // 0 .. 2^24 - 1
  float lg;
  if (t >= (1u << 23))
    lg = log1pf(-(float)((1u << 24) - 1u - t) * 0x1p-24f);
  else
    lg = logf(((float)t + 1.0f) * 0x1p-24f);
  const float rad = sqrtf(-2.0f * lg);
  const float two_u2 = (float)(2u * (y >> 9) + 1u) * 0x1p-23f;  // 2 u2, exact
  float sn, cs;
  sincospif(two_u2, &sn, &cs);
  z0 = rad * cs;
  z1 = rad * sn;
}

__global__ void philox_words_kernel(uint64_t seed, uint32_t sid, int64_t n_blocks, uint4* out) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < n_blocks;
       n += (int64_t)gridDim.x * blockDim.x)
    out[n] = philox_block(seed, sid, (uint64_t)n);
}

// One thread per Philox block (4 consecutive elements of the row-major
// rows x cols matrix, element e = i*cols + j), written at row stride ldo.
__global__ void gaussian_kernel(uint64_t seed, uint32_t sid, int64_t rows, int64_t cols,
                                float* __restrict__ out, int64_t ldo) {
  const int64_t total = rows * cols;
  const int64_t nb = (total + 3) / 4;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < nb;
       n += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = philox_block(seed, sid, (uint64_t)n);
    float z[4];
    box_muller(w.x, w.y, z[0], z[1]);
    box_muller(w.z, w.w, z[2], z[3]);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t e = 4 * n + u;
      if (e < total) {
        const int64_t i = e / cols, j = e - i * cols;
        out[i * ldo + j] = z[u];
      }
    }
  }
}

static int grid_for(int64_t work, int threads) {
  int64_t g = ceil_div(work, threads);
  if (g > num_sms() * 32) g = num_sms() * 32;
  if (g < 1) g = 1;
  return (int)g;
}

lramm_status launch_philox_words(uint64_t seed, uint32_t sid, int64_t n_blocks, uint32_t* out,
                                 cudaStream_t s) {
  if (n_blocks <= 0) return LRAMM_OK;
  philox_words_kernel<<<grid_for(n_blocks, 256), 256, 0, s>>>(seed, sid, n_blocks,
                                                               reinterpret_cast<uint4*>(out));
  return last_launch();
}

lramm_status launch_gaussian(uint64_t seed, uint32_t sid, int64_t rows, int64_t cols, float* out,
                             int64_t ldo, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return LRAMM_OK;
  gaussian_kernel<<<grid_for(ceil_div(rows * cols, 4), 256), 256, 0, s>>>(seed, sid, rows, cols,
                                                                          out, ldo);
  return last_launch();
}

}  // namespace lramm
