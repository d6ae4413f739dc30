// philox.cuh -- Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11), used as the uniform draw of the delay process of Sec. 5.1.
// Host and device share this definition so every delay the kernels draw can be replayed on the host.
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define AT_HD __host__ __device__ __forceinline__
#else
#define AT_HD inline
#endif

namespace atfd {

struct U32x4 {
  uint32_t v[4];
};

AT_HD void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo) {
#if defined(__CUDA_ARCH__)
  *lo = a * b;
  *hi = __umulhi(a, b);
#else
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *lo = (uint32_t)p;
  *hi = (uint32_t)(p >> 32);
#endif
}

// ten rounds; the key schedule adds the two Weyl constants between rounds
AT_HD U32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
  const uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
  const uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(kMul0, c0, &hi0, &lo0);
    mulhilo32(kMul1, c2, &hi1, &lo1);
    const uint32_t y0 = hi1 ^ c1 ^ k0;
    const uint32_t y2 = hi0 ^ c3 ^ k1;
    c0 = y0;
    c1 = lo1;
    c2 = y2;
    c3 = lo0;
    k0 += kWeyl0;
    k1 += kWeyl1;
  }
  U32x4 r;
  r.v[0] = c0; r.v[1] = c1; r.v[2] = c2; r.v[3] = c3;
  return r;
}

// Raw delay of PE side `side` at step `step`: counter (step, side, 0, 0), key = seed.  The 32-bit word
// x0 stands for the uniform draw x0 / 2^32; bins are uniform (thr == nullptr) or given by L-1 ascending
// integer edges on [0, 2^32].
AT_HD int delay_draw(uint64_t seed, uint32_t step, uint32_t side, int L, const uint64_t *thr) {
  const U32x4 x = philox4x32_10(step, side, 0u, 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint32_t x0 = x.v[0];
  if (thr == nullptr) return (int)(((uint64_t)x0 * (uint64_t)(uint32_t)L) >> 32);
  int k = 0;
  for (int m = 0; m + 1 < L; ++m) k += ((uint64_t)x0 >= thr[m]) ? 1 : 0;
  return k;
}

// Levels before 0 do not exist: a scheme reading T successive levels n-k..n-k-T+1 can use at most
// k = n-(T-1); a zero delay reads level n only.
AT_HD int delay_clamp(int k, int64_t n, int T) {
  if (k <= 0) return 0;
  int64_t lim = n - (int64_t)(T - 1);
  if (lim < 0) lim = 0;
  return (int64_t)k < lim ? k : (int)lim;
}

}  // namespace atfd
