// fwd.cu -- the fused forward step of the asynchrony-tolerant (AT) scheme on sm_103a.
//
// One launch advances U^n -> U^{n+1} by forward Euler (Sec. 4.1, Eq. "time_disc" with one level):
//     U^{n+1}_i = U^n_i + dt sum_a ( -c_a D1_a U + alpha D2_a U )_i
// with the central differences and the AT tables folded into merged per-axis coefficients
//     s_{a,j} = dt ( -c_a cd1_j / dx_a + alpha cd2_j / dx_a^2 ),   s0 = 1 + sum_a s_{a,0},
// so an interior point costs one multiply and 2*h*dim fused multiply-adds.
//
// Points within h of a PE boundary (the set I_B of Sec. 2) read, for each stencil point across that
// boundary (a buffer point), the extrapolated halo value
//     u~ = sum_{m<T} w_m(k) U^{n-k-m}                                   (k = that side's delay)
// where w_m(k) are the stage-2 weights of Example 3.  Since sum_m w_m(k) CD(.. U^{n-k-m} ..) =
// CD(.. u~ ..) for the time-expanded tables ((1,2,2)b, (2,2,2)b, (1,4,2), (2,4,2)), the halo value is
// formed once and shared by the first- and second-derivative taps.  The delay k of every PE side is
// drawn in-kernel from Philox (Sec. 5.1) keyed by (seed, step, side) and clamped so that no level before
// 0 is read; one designated thread per side writes the raw draw to the delay log.
//
// The kernel is FP64-FMA bound on GB300 (2 FP64 FMA lanes per SM per clock): loads go through L1, the
// DFMA chain per point is the minimum 1 + 2 h dim operations.
#include "internal.h"
#include "philox.cuh"

namespace {

__device__ __forceinline__ int wrap_coord(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Halo value of `cell` seen across a PE side with effective delay k (T successive levels).
__device__ __forceinline__ double halo_value(const StepParams &p, int64_t cell, int64_t n, int k) {
  if (k == 0) return __ldg(p.ring + (n % p.R) * p.ntot + cell);
  double acc = 0.0;
#pragma unroll
  for (int m = 0; m < AT_MAX_T; ++m) {
    if (m >= p.T) break;
    const int64_t lev = n - k - m;
    acc = fma(p.w[k][m], __ldg(p.ring + (lev % p.R) * p.ntot + cell), acc);
  }
  return acc;
}

template <int DIM, int H>
__global__ void __launch_bounds__(256) forward_step_kernel(const StepParams p, const int64_t n) {
  const double *__restrict__ un = p.ring + (n % p.R) * p.ntot;
  double *__restrict__ out = p.ring + ((n + 1) % p.R) * p.ntot;
  const int nx = p.n[0], ny = DIM == 3 ? p.n[1] : 1;
  const int64_t stride[3] = {1, (int64_t)nx, (int64_t)nx * ny};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.ntot;
       i += (int64_t)gridDim.x * blockDim.x) {
    int c[3];
    if (DIM == 1) {
      c[0] = (int)i; c[1] = 0; c[2] = 0;
    } else {
      const int64_t yz = i / nx;
      c[0] = (int)(i - yz * nx);
      c[2] = (int)(yz / ny);
      c[1] = (int)(yz - (int64_t)c[2] * ny);
    }
    int pos[3], pidx[3];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      pidx[a] = c[a] / p.S[a];
      pos[a] = c[a] - pidx[a] * p.S[a];
    }
    double acc = p.s0 * __ldg(un + i);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int S = p.S[a];
      const bool lo = pos[a] < H, hi = pos[a] >= S - H;
      const bool edge = p.use_pe[a] && (lo || hi);
      int k = 0;
      if (lo || hi) {
        int pe_id = pidx[0];
        if (DIM == 3) pe_id = (pidx[2] * p.pe[1] + pidx[1]) * p.pe[0] + pidx[0];
        const int64_t side = 2 * (int64_t)DIM * pe_id + 2 * a + (lo ? 0 : 1);
        int raw = 0;
        if (p.scheme != 0) raw = atfd::delay_draw(p.seed, (uint32_t)n, (uint32_t)side, p.L, p.use_thr ? p.thr : nullptr);
        k = atfd::delay_clamp(raw, n, p.T);
        // the log writer of this side: the edge point of the side with the other coordinates at the PE origin
        bool writer = lo ? (pos[a] == 0) : (pos[a] == S - 1);
#pragma unroll
        for (int b = 0; b < DIM; ++b)
          if (b != a && pos[b] != 0) writer = false;
        if (writer && p.log != nullptr) p.log[n * p.nb + side] = (uint8_t)raw;
      }
#pragma unroll
      for (int j = -H; j <= H; ++j) {
        if (j == 0) continue;
        const int cj = wrap_coord(c[a] + j, p.n[a]);
        const int64_t cell = i + (int64_t)(cj - c[a]) * stride[a];
        double v;
        if (edge && (pos[a] + j < 0 || pos[a] + j >= S))
          v = halo_value(p, cell, n, k);
        else
          v = __ldg(un + cell);
        acc = fma(p.s[a][j + H], v, acc);
      }
    }
    out[i] = acc;
  }
}

}  // namespace

cudaError_t launch_forward_step(const StepParams &p, int64_t n, cudaStream_t st) {
  const int threads = 256;
  int64_t blocks = (p.ntot + threads - 1) / threads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (p.dim == 1) {
    if (p.h == 1) forward_step_kernel<1, 1><<<(int)blocks, threads, 0, st>>>(p, n);
    else forward_step_kernel<1, 2><<<(int)blocks, threads, 0, st>>>(p, n);
  } else {
    if (p.h == 1) forward_step_kernel<3, 1><<<(int)blocks, threads, 0, st>>>(p, n);
    else forward_step_kernel<3, 2><<<(int)blocks, threads, 0, st>>>(p, n);
  }
  return cudaGetLastError();
}
