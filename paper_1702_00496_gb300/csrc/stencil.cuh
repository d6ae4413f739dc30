// stencil.cuh -- device building blocks of the fused AT step, shared by the per-step kernels (fwd.cu) and
// the persistent ensemble kernel (ensemble.cu).  See fwd.cu for the method and its citations.
#pragma once
#include "internal.h"
#include "philox.cuh"

namespace atfd {

// Load policies.  LdgNC reads through the non-coherent read-only path: legal in the per-step kernels, whose
// read slots are never written during the launch.  LdCoherent is a plain load, for kernels that read back what
// they wrote earlier in the same launch (after a barrier).
struct LdgNC {
  static __device__ __forceinline__ double ld(const double *p) { return __ldg(p); }
  static __device__ __forceinline__ double2 ld2(const double *p) { return __ldg(reinterpret_cast<const double2 *>(p)); }
};
struct LdCoherent {
  static __device__ __forceinline__ double ld(const double *p) { return *p; }
  static __device__ __forceinline__ double2 ld2(const double *p) { return *reinterpret_cast<const double2 *>(p); }
};


__device__ __forceinline__ int wrap_coord(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Halo value of `cell` seen across a PE side with effective delay k (T successive levels).
template <class LD>
__device__ __forceinline__ double halo_value(const StepParams &p, int64_t cell, int64_t n, int k) {
  if (k == 0) return LD::ld(p.ring + (n % p.R) * p.ntot + cell);
  double acc = 0.0;
#pragma unroll
  for (int m = 0; m < AT_MAX_T; ++m) {
    if (m >= p.T) break;
    const int64_t lev = n - k - m;
    acc = fma(p.w[k][m], LD::ld(p.ring + (lev % p.R) * p.ntot + cell), acc);
  }
  return acc;
}

// Updated value of point i (linear index) with coordinates c: the general path, used for points within h
// of a PE edge, points whose stencil wraps around the periodic domain, and ragged groups.
template <int DIM, int H, class LD>
__device__ __noinline__ double point_update(const StepParams &p, const double *__restrict__ un, int64_t n, int64_t i,
                                            const int c[3]) {
  const int64_t stride[3] = {1, (int64_t)p.n[0], (int64_t)p.n[0] * p.n[1]};
  int pos[3], pidx[3];
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    pidx[a] = c[a] / p.S[a];
    pos[a] = c[a] - pidx[a] * p.S[a];
  }
  double acc = fma(p.s0, LD::ld(un + i), p.zero);
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
        v = halo_value<LD>(p, cell, n, k);
      else
        v = LD::ld(un + cell);
      acc = fma(p.s[a][j + H], v, acc);
    }
  }
  return acc;
}


// Merged stencil of one point from the values of its line along one axis (v[H + j] = u_{i+j}).
template <int H>
__device__ __forceinline__ double axis_taps(const double (&s)[2 * AT_MAX_H + 1], const double *v, double acc) {
#pragma unroll
  for (int j = -H; j <= H; ++j)
    if (j != 0) acc = fma(s[j + H], v[H + j], acc);
  return acc;
}

// One group of four consecutive 1D points starting at i0 (a multiple of 4): the straight FMA path with four
// independent chains when the group lies inside one PE, at least h from its edges and from the ends of the
// domain; otherwise the general path point by point.  Requires N even and a 16-byte aligned slot.
template <int H, class LD>
__device__ __forceinline__ void group_1d(const StepParams &p, const double *__restrict__ un, double *__restrict__ out,
                                         int64_t n, int i0) {
  const int N = p.n[0], S = p.S[0];
  const int pos0 = i0 % S;
  const bool inside = (i0 >= 2) && (i0 + 6 <= N) && (!p.use_pe[0] || (pos0 >= H && pos0 + 3 < S - H));
  if (inside) {
    const double2 a = LD::ld2(un + i0 - 2), b = LD::ld2(un + i0), c = LD::ld2(un + i0 + 2), d = LD::ld2(un + i0 + 4);
    const double v[8] = {a.x, a.y, b.x, b.y, c.x, c.y, d.x, d.y};  // u[i0-2 .. i0+5]
    double r[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) r[q] = axis_taps<H>(p.s[0], v + q + 2 - H, fma(p.s0, v[q + 2], p.zero));
    reinterpret_cast<double2 *>(out + i0)[0] = make_double2(r[0], r[1]);
    reinterpret_cast<double2 *>(out + i0)[1] = make_double2(r[2], r[3]);
  } else {
    for (int q = 0; q < 4 && i0 + q < N; ++q) {
      const int c[3] = {i0 + q, 0, 0};
      out[i0 + q] = point_update<1, H, LD>(p, un, n, i0 + q, c);
    }
  }
}

}  // namespace atfd
