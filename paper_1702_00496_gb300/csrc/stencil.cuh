// stencil.cuh -- device building blocks of the fused AT step, shared by the per-step kernels (fwd.cu) and the
// persistent ensemble kernel (ensemble.cu).
//
// A thread updates a group of four consecutive x points (x0 a multiple of 4) of one (y, z) row.  It loads
// the level-n values its merged stencil needs -- the x window x0-W .. x0+3+W (W = h rounded up to even, so the
// window starts on 16 bytes) and, in 3D, the four values of rows y +- j and z +- j -- and replaces every value
// that lies outside the group's PE (a buffer point, Sec. 2) by the halo value its PE side sees:
//     u~ = sum_{m<T} w_m(k) U^{n-k-m}     (k: that side's effective delay for step n; k = 0 keeps U^n)
// Groups never straddle a PE (PE widths are multiples of 4 on these paths), so each loaded value is either
// inside the PE or a buffer point of exactly one side.  The update is then the same chain of FMAs for every
// group:  r = fma(s0, u_i, +0), the taps of axis x in offset order, then axis y, then axis z.
//
// With Adams-Bashforth time stepping (Sec. 4.1, Eq. "time_disc" with two or three levels) the same chain,
// without the 1 in s0, gives dt f^n; the update adds the stored dt f^{n-1}, dt f^{n-2} with their weights and
// keeps dt f^n in place of the oldest one.
//
// Delays are drawn once per PE side and step (Philox, Sec. 5.1) by a draw pass into a small array of
// effective delays (uint8, clamped so that no level before 0 is read); the raw draw goes to the delay log.
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

// Draw the delays of step n for sides b = first, first+stride, ...: effective delay to keff[b], raw draw to
// the log row n (when the log holds that row).
__device__ __forceinline__ void draw_sides(const StepParams &p, int64_t n, int64_t first, int64_t stride,
                                           uint8_t *keff) {
  for (int64_t b = first; b < p.nb; b += stride) {
    int raw = 0;
    if (p.scheme != 0) raw = delay_draw(p.seed, (uint32_t)n, (uint32_t)b, p.L, p.use_thr ? p.thr : nullptr);
    keff[b] = (uint8_t)delay_clamp(raw, n, p.T);
    if (p.log != nullptr && n < p.log_steps) p.log[n * p.nb + b] = (uint8_t)raw;
  }
}

// Slot of the level `back` levels below the level in slot sn (0 <= back < R): no 64-bit modulo per load.
__device__ __forceinline__ int64_t slot_back(int sn, int back, int R) {
  const int s = sn - back;
  return s < 0 ? s + R : s;
}

// Halo value of `cell` seen across a PE side with effective delay k >= 1 (T successive levels); sn is the
// slot of level n.
template <class LD>
__device__ __forceinline__ double halo_value(const StepParams &p, int64_t cell, int sn, int k) {
  double acc = fma(p.w[k][0], LD::ld(p.ring + slot_back(sn, k, p.R) * p.ntot + cell), p.zero);
#pragma unroll
  for (int m = 1; m < AT_MAX_T; ++m) {
    if (m >= p.T) break;
    acc = fma(p.w[k][m], LD::ld(p.ring + slot_back(sn, k + m, p.R) * p.ntot + cell), acc);
  }
  return acc;
}

// Order of the 1D groups that keeps the lanes of a warp on one path: the interior groups of every PE (local
// index 1 .. gS-2 of the gS = S/4 groups of a PE) first, then the two edge groups of every PE.  Any order is
// correct; this one avoids warps in which a few lanes take the halo path.  k < number of groups.
__device__ __forceinline__ int64_t group_1d_order(const StepParams &p, int64_t k) {
  const uint32_t gS = (uint32_t)(p.use_pe[0] ? p.S[0] >> 2 : p.n[0] >> 2);
  if (gS < 3) return k;
  const uint32_t inner = gS - 2, npe = (uint32_t)(p.n[0] >> 2) / gS, uk = (uint32_t)k;
  const uint32_t n_int = npe * inner;
  if (uk < n_int) {
    const uint32_t pe = uk / inner;
    return (int64_t)pe * gS + 1 + (uk - pe * inner);
  }
  const uint32_t kk = uk - n_int;
  return (int64_t)(kk >> 1) * gS + ((kk & 1) ? gS - 1 : 0);
}

// The same order with e edge groups at each PE end (e = 1 is group_1d_order): the gS - 2e inner groups of every PE
// first, then the 2e edge groups of every PE.  k < number of groups; requires gS > 2e.
__device__ __forceinline__ int64_t group_1d_order_e(const StepParams &p, int64_t k, int e) {
  const uint32_t gS = (uint32_t)(p.use_pe[0] ? p.S[0] >> 2 : p.n[0] >> 2);
  if (e == 0) return k;
  const uint32_t inner = gS - 2 * e, npe = (uint32_t)(p.n[0] >> 2) / gS, uk = (uint32_t)k;
  const uint32_t n_int = npe * inner;
  if (uk < n_int) {
    const uint32_t pe = uk / inner;
    return (int64_t)pe * gS + e + (uk - pe * inner);
  }
  const uint32_t kk = uk - n_int, pe = kk / (2 * e), r = kk - pe * (2 * e);
  return (int64_t)pe * gS + (r < (uint32_t)e ? r : gS - 2 * e + r);
}

// Side index of face (axis a, lo/hi) of the PE with index (px, py, pz).
template <int DIM>
__device__ __forceinline__ int64_t side_of(const StepParams &p, const int pidx[3], int a, int hi) {
  int64_t pe = pidx[0];
  if (DIM == 3) pe = ((int64_t)pidx[2] * p.pe[1] + pidx[1]) * p.pe[0] + pidx[0];
  return 2 * (int64_t)DIM * pe + 2 * a + hi;
}

// Half-width of the x window of a group: h rounded up to an even count, so the window's loads start on 16 bytes.
template <int H>
struct XWin {
  static constexpr int W = (H + 1) / 2 * 2;
  static constexpr int N = 4 + 2 * W;
};

// The merged stencil of the four points x0..x0+3 of row (y, z) into r[4] (and their level-n values into uc[4]);
// requires n[0] % 4 == 0 and a 16-byte aligned slot.  keff: effective delays of step n.  ALPHA = true evaluates
// the alpha derivative of the step instead (coefficients q0, q: dt times the AT second derivative).  OWN_SIDES = true
// reads the delay of an x side only when the group reaches that side's buffer points (for callers whose other
// sides' delays may be in flight).
template <int DIM, int H, class LD, bool ALPHA, bool OWN_SIDES = false>
__device__ __forceinline__ void group_eval(const StepParams &p, const uint8_t *__restrict__ keff,
                                           const double *__restrict__ un, int64_t n, int x0, int y, int z,
                                           double r[4], double uc[4]) {
  constexpr int W = XWin<H>::W, NW = XWin<H>::N;
  const int nx = p.n[0];
  const int sn = (int)(n % p.R);
  const int64_t row = DIM == 3 ? ((int64_t)z * p.n[1] + y) * nx : 0;
  const int64_t i0 = row + x0;
  int pidx[3] = {x0 / p.S[0], 0, 0}, pos[3] = {0, 0, 0};
  pos[0] = x0 - pidx[0] * p.S[0];
  if (DIM == 3) {
    pidx[1] = y / p.S[1]; pos[1] = y - pidx[1] * p.S[1];
    pidx[2] = z / p.S[2]; pos[2] = z - pidx[2] * p.S[2];
  }
  // x window: cells x0-W .. x0+3+W of the row
  double v[NW];
  if (x0 >= W && x0 + 4 + W <= nx) {
#pragma unroll
    for (int t = 0; t < NW; t += 2) {
      const double2 a = LD::ld2(un + i0 - W + t);
      v[t] = a.x; v[t + 1] = a.y;
    }
  } else {
#pragma unroll
    for (int t = 0; t < NW; ++t) v[t] = LD::ld(un + row + wrap_coord(x0 - W + t, nx));
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) uc[q] = v[W + q];
  if (p.use_pe[0] && (pos[0] < H || pos[0] + 3 >= p.S[0] - H)) {
    const bool lo = !OWN_SIDES || pos[0] < H, hi = !OWN_SIDES || pos[0] + 3 >= p.S[0] - H;
    const int kl = lo ? keff[side_of<DIM>(p, pidx, 0, 0)] : 0, kr = hi ? keff[side_of<DIM>(p, pidx, 0, 1)] : 0;
#pragma unroll
    for (int t = W - H; t <= W + 3 + H; ++t) {
      const int rel = pos[0] - W + t;
      const int k = rel < 0 ? kl : (rel >= p.S[0] ? kr : 0);
      if (k > 0) v[t] = halo_value<LD>(p, row + wrap_coord(x0 - W + t, nx), sn, k);
    }
  }
  const double c0 = ALPHA ? p.q0 : p.s0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double acc = fma(c0, v[q + W], p.zero);
#pragma unroll
    for (int j = -H; j <= H; ++j)
      if (j != 0) acc = fma(ALPHA ? p.q[0][j + H] : p.s[0][j + H], v[q + W + j], acc);
    r[q] = acc;
  }
  if (DIM == 3) {
#pragma unroll
    for (int a = 1; a < 3; ++a) {
      const int c = a == 1 ? y : z, na = p.n[a];
      const int64_t st = a == 1 ? (int64_t)nx : (int64_t)nx * p.n[1];
      const bool edge = p.use_pe[a] && (pos[a] < H || pos[a] >= p.S[a] - H);
      int kl = 0, kr = 0;
      if (edge) {
        kl = keff[side_of<DIM>(p, pidx, a, 0)];
        kr = keff[side_of<DIM>(p, pidx, a, 1)];
      }
#pragma unroll
      for (int j = -H; j <= H; ++j) {
        if (j == 0) continue;
        const int cj = wrap_coord(c + j, na);
        const int64_t base = i0 + (int64_t)(cj - c) * st;
        const int k = !edge ? 0 : (pos[a] + j < 0 ? kl : (pos[a] + j >= p.S[a] ? kr : 0));
        double w[4];
        if (k > 0) {
#pragma unroll
          for (int q = 0; q < 4; ++q) w[q] = halo_value<LD>(p, base + q, sn, k);
        } else {
          const double2 e = LD::ld2(un + base), f = LD::ld2(un + base + 2);
          w[0] = e.x; w[1] = e.y; w[2] = f.x; w[3] = f.y;
        }
        const double s = ALPHA ? p.q[a][j + H] : p.s[a][j + H];
#pragma unroll
        for (int q = 0; q < 4; ++q) r[q] = fma(s, w[q], r[q]);
      }
    }
  }
}

// NP consecutive stored right-hand sides (16-byte aligned for NP > 1).
template <int NP>
__device__ __forceinline__ void ab_load(const double *src, double a[NP]) {
  if constexpr (NP == 1) {
    a[0] = src[0];
  } else {
#pragma unroll
    for (int q = 0; q < NP; q += 2) {
      const double2 v = *reinterpret_cast<const double2 *>(src + q);
      a[q] = v.x; a[q + 1] = v.y;
    }
  }
}

template <int NP>
__device__ __forceinline__ void ab_store(double *dst, const double a[NP]) {
  if constexpr (NP == 1) {
    dst[0] = a[0];
  } else {
#pragma unroll
    for (int q = 0; q < NP; q += 2) *reinterpret_cast<double2 *>(dst + q) = make_double2(a[q], a[q + 1]);
  }
}

// Adams-Bashforth combination of NP consecutive points starting at i (16-byte aligned for NP = 4): r holds
// dt f^n and becomes U^{n+1} = U^n + sum_{m<l} beta_m dt f^{n-m} (l = levels stored so far, at most ts), formed
// as a chain of l FMAs onto U^n; dt f^n takes the slot of the oldest right-hand side, which only this thread
// reads, after the read.
//
// STEADY = true: the host launches this form only for steps whose ts levels are all stored (l = ts); with ts = 2
// the weights beta[1] are then fixed and come straight from the kernel parameters.  The operations are the same;
// this takes Case 4 (AB2, N = 2^24) on GB300 from 248 to 214 us per step.  (AB3 in this form ran at 492 against
// 307 us, so other ts take the general code.)
template <int NP, bool STEADY = false>
__device__ __forceinline__ void ab_combine(const StepParams &p, int64_t n, int64_t i, const double u[NP],
                                           double r[NP]) {
  if (STEADY && p.ts == 2) {
    double *f = p.frhs + i;  // dt f^{n-1}, then dt f^n
    double a1[NP];
    ab_load<NP>(f, a1);
    ab_store<NP>(f, r);
#pragma unroll
    for (int q = 0; q < NP; ++q) r[q] = fma(p.beta[1][0], r[q], u[q]);
#pragma unroll
    for (int q = 0; q < NP; ++q) r[q] = fma(p.beta[1][1], a1[q], r[q]);
    return;
  }
  const int64_t stored = n - *p.ab_first + 1;
  const int l = stored < p.ts ? (int)stored : p.ts;
  const double *beta = p.beta[l - 1];
  const bool two = p.ts == 3;  // two stored slots, else one
  double *f_now = p.frhs + (two ? (n & 1) : 0) * p.ntot + i;          // dt f^{n-2} (AB3) or dt f^{n-1} (AB2)
  const double *f_1 = p.frhs + (two ? ((n - 1) & 1) : 0) * p.ntot + i;  // dt f^{n-1}
  double a1[NP], a2[NP];
  if (l > 1) ab_load<NP>(f_1, a1);
  if (l > 2) ab_load<NP>(f_now, a2);
  ab_store<NP>(f_now, r);
#pragma unroll
  for (int q = 0; q < NP; ++q) r[q] = fma(beta[0], r[q], u[q]);
  if (l > 1) {
#pragma unroll
    for (int q = 0; q < NP; ++q) r[q] = fma(beta[1], a1[q], r[q]);
  }
  if (l > 2) {
#pragma unroll
    for (int q = 0; q < NP; ++q) r[q] = fma(beta[2], a2[q], r[q]);
  }
}

// Update the four points x0..x0+3 of row (y, z) (the forward step; AB: 0 forward Euler, 1 Adams-Bashforth, 2
// AB2 with both levels stored, ab_combine's STEADY form).
template <int DIM, int H, class LD, int AB = 0, bool OWN_SIDES = false>
__device__ __forceinline__ void group_update(const StepParams &p, const uint8_t *__restrict__ keff,
                                             const double *__restrict__ un, double *__restrict__ out, int64_t n,
                                             int x0, int y, int z) {
  double r[4], uc[4];
  group_eval<DIM, H, LD, false, OWN_SIDES>(p, keff, un, n, x0, y, z, r, uc);
  const int64_t i0 = (DIM == 3 ? ((int64_t)z * p.n[1] + y) * p.n[0] : 0) + x0;
  if (AB) ab_combine<4, AB == 2>(p, n, i0, uc, r);
  reinterpret_cast<double2 *>(out + i0)[0] = make_double2(r[0], r[1]);
  reinterpret_cast<double2 *>(out + i0)[1] = make_double2(r[2], r[3]);
}

// One point of any shape (the fallback for point counts that are not a multiple of 4), same arithmetic.
template <int DIM, int H, class LD>
__device__ double point_update(const StepParams &p, const uint8_t *__restrict__ keff, const double *__restrict__ un,
                               int64_t n, int64_t i, const int c[3]) {
  const int64_t stride[3] = {1, (int64_t)p.n[0], (int64_t)p.n[0] * p.n[1]};
  int pos[3] = {0, 0, 0}, pidx[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    pidx[a] = c[a] / p.S[a];
    pos[a] = c[a] - pidx[a] * p.S[a];
  }
  double acc = fma(p.s0, LD::ld(un + i), p.zero);
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const bool edge = p.use_pe[a] && (pos[a] < H || pos[a] >= p.S[a] - H);
#pragma unroll
    for (int j = -H; j <= H; ++j) {
      if (j == 0) continue;
      const int cj = wrap_coord(c[a] + j, p.n[a]);
      const int64_t cell = i + (int64_t)(cj - c[a]) * stride[a];
      int k = 0;
      if (edge && pos[a] + j < 0) k = keff[side_of<DIM>(p, pidx, a, 0)];
      if (edge && pos[a] + j >= p.S[a]) k = keff[side_of<DIM>(p, pidx, a, 1)];
      const double v = k > 0 ? halo_value<LD>(p, cell, (int)(n % p.R), k) : LD::ld(un + cell);
      acc = fma(p.s[a][j + H], v, acc);
    }
  }
  return acc;
}

// Viscous Burgers' equation (1D, Case 6): dt f = -u_i (dt D1 u) + dt alpha D2 u with the same x window and the
// same extrapolated halo values as the linear step; r receives dt f^n of the four points x0..x0+3, uc their
// level-n values.  Each derivative is its own FMA chain; u_i enters through the final FMA.
template <int H, class LD>
__device__ __forceinline__ void group_eval_burgers(const StepParams &p, const uint8_t *__restrict__ keff,
                                                   const double *__restrict__ un, int64_t n, int x0, double r[4],
                                                   double uc[4]) {
  constexpr int W = XWin<H>::W, NW = XWin<H>::N;
  const int nx = p.n[0];
  const int sn = (int)(n % p.R);
  const int pidx[3] = {x0 / p.S[0], 0, 0};
  const int pos0 = x0 - pidx[0] * p.S[0];
  double v[NW];
  if (x0 >= W && x0 + 4 + W <= nx) {
#pragma unroll
    for (int t = 0; t < NW; t += 2) {
      const double2 a = LD::ld2(un + x0 - W + t);
      v[t] = a.x; v[t + 1] = a.y;
    }
  } else {
#pragma unroll
    for (int t = 0; t < NW; ++t) v[t] = LD::ld(un + wrap_coord(x0 - W + t, nx));
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) uc[q] = v[W + q];
  if (p.use_pe[0] && (pos0 < H || pos0 + 3 >= p.S[0] - H)) {
    const int kl = keff[side_of<1>(p, pidx, 0, 0)], kr = keff[side_of<1>(p, pidx, 0, 1)];
#pragma unroll
    for (int t = W - H; t <= W + 3 + H; ++t) {
      const int rel = pos0 - W + t;
      const int k = rel < 0 ? kl : (rel >= p.S[0] ? kr : 0);
      if (k > 0) v[t] = halo_value<LD>(p, wrap_coord(x0 - W + t, nx), sn, k);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double a1 = fma(p.b1[0], v[q + W - H], p.zero);
    double a2 = fma(p.b2[H], v[q + W], p.zero);
#pragma unroll
    for (int j = -H; j <= H; ++j) {
      if (j == 0) continue;
      if (j != -H) a1 = fma(p.b1[j + H], v[q + W + j], a1);
      a2 = fma(p.b2[j + H], v[q + W + j], a2);
    }
    r[q] = fma(-v[q + W], a1, a2);
  }
}

// One point of the Burgers step (per-point shapes): dt f^n of point i.
template <int H, class LD>
__device__ double point_update_burgers(const StepParams &p, const uint8_t *__restrict__ keff,
                                       const double *__restrict__ un, int64_t n, int64_t i) {
  const int c = (int)i;
  const int pidx[3] = {c / p.S[0], 0, 0};
  const int pos = c - pidx[0] * p.S[0];
  const bool edge = p.use_pe[0] && (pos < H || pos >= p.S[0] - H);
  const double ui = LD::ld(un + i);
  double a1 = p.zero;
  double a2 = fma(p.b2[H], ui, p.zero);
#pragma unroll
  for (int j = -H; j <= H; ++j) {
    if (j == 0) continue;
    const int cj = wrap_coord(c + j, p.n[0]);
    int k = 0;
    if (edge && pos + j < 0) k = keff[side_of<1>(p, pidx, 0, 0)];
    if (edge && pos + j >= p.S[0]) k = keff[side_of<1>(p, pidx, 0, 1)];
    const double v = k > 0 ? halo_value<LD>(p, cj, (int)(n % p.R), k) : LD::ld(un + cj);
    a1 = j == -H ? fma(p.b1[0], v, p.zero) : fma(p.b1[j + H], v, a1);
    a2 = fma(p.b2[j + H], v, a2);
  }
  return fma(-ui, a1, a2);
}

// Rows expanded in space (AT_AT_SPACE2 / AT_AT_SPACE1, order 2): a point at the edge of its PE along a split axis
// (position 0 or S-1) whose side has delay k > 0 takes that axis's edge row -- in-PE taps at level n, buffer taps
// at level n-k -- instead of the central taps; every other axis and point keeps the central difference.  One
// point, any shape; the same FMA chain order as the central path (centre first, then axis by axis).
template <int DIM, class LD>
__device__ double point_update_space(const StepParams &p, const uint8_t *__restrict__ keff,
                                     const double *__restrict__ un, int64_t n, int64_t i, const int c[3]) {
  const int64_t stride[3] = {1, (int64_t)p.n[0], (int64_t)p.n[0] * p.n[1]};
  const int sn = (int)(n % p.R);
  int pidx[3] = {0, 0, 0}, krow[3] = {0, 0, 0}, srow[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < DIM; ++a) pidx[a] = c[a] / p.S[a];  // the whole PE index before any side lookup
  double c0 = p.ts > 1 ? 0.0 : 1.0;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const int pos = c[a] - pidx[a] * p.S[a];
    if (p.use_pe[a] && (pos == 0 || pos == p.S[a] - 1)) {
      srow[a] = pos == 0 ? 0 : 1;
      krow[a] = keff[side_of<DIM>(p, pidx, a, srow[a])];
    }
    if (krow[a] == 0) c0 += p.sc[a];
  }
  double acc = fma(c0, LD::ld(un + i), p.zero);
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    if (krow[a] > 0) {
      const int s = srow[a], nt = p.ecount[a][s];
      for (int t = 0; t < nt; ++t) {
        const int cj = wrap_coord(c[a] + p.ej[a][s][t], p.n[a]);
        const int64_t cell = i + (int64_t)(cj - c[a]) * stride[a];
        const double *lvl = p.ebuf[a][s][t] ? p.ring + slot_back(sn, krow[a], p.R) * p.ntot : un;
        acc = fma(p.ec[a][s][t], LD::ld(lvl + cell), acc);
      }
    } else {
#pragma unroll
      for (int j = -1; j <= 1; j += 2) {
        const int cj = wrap_coord(c[a] + j, p.n[a]);
        acc = fma(p.s[a][j + 1], LD::ld(un + i + (int64_t)(cj - c[a]) * stride[a]), acc);
      }
    }
  }
  return acc;
}

// Does the group x0..x0+3 of row (y, z) hold a PE-edge point of a split axis (AT_AT_SPACE2 / AT_AT_SPACE1)?
template <int DIM>
__device__ __forceinline__ bool group_at_space_edge(const StepParams &p, int x0, int y, int z) {
  if (p.use_pe[0]) {
    const int pos = x0 % p.S[0];
    if (pos == 0 || pos + 4 == p.S[0]) return true;
  }
  if (DIM == 3) {
    if (p.use_pe[1]) {
      const int pos = y % p.S[1];
      if (pos == 0 || pos == p.S[1] - 1) return true;
    }
    if (p.use_pe[2]) {
      const int pos = z % p.S[2];
      if (pos == 0 || pos == p.S[2] - 1) return true;
    }
  }
  return false;
}

// One group of the forward step for every scheme: groups holding a PE-edge point of a scheme expanded in space
// go point by point through its edge rows, all others through the grouped central / time-expanded path.  KIND
// selects the kernel variant -- 0: central and time-expanded rows, 1: Burgers' equation (1D), 2: rows expanded in
// space -- so each kernel carries only its own path.
template <int DIM, int H, class LD, int AB, int KIND = 0>
__device__ __forceinline__ void group_step(const StepParams &p, const uint8_t *__restrict__ keff,
                                           const double *__restrict__ un, double *__restrict__ out, int64_t n,
                                           int x0, int y, int z) {
  if (DIM == 1 && KIND == 1) {
    double r[4], uc[4];
    group_eval_burgers<H, LD>(p, keff, un, n, x0, r, uc);
    if (AB) {
      ab_combine<4, AB == 2>(p, n, x0, uc, r);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) r[q] = uc[q] + r[q];
    }
    reinterpret_cast<double2 *>(out + x0)[0] = make_double2(r[0], r[1]);
    reinterpret_cast<double2 *>(out + x0)[1] = make_double2(r[2], r[3]);
    return;
  }
  if (KIND == 2 && H == 1 && !AB && group_at_space_edge<DIM>(p, x0, y, z)) {
    const int64_t i0 = (DIM == 3 ? ((int64_t)z * p.n[1] + y) * p.n[0] : 0) + x0;
    int c[3] = {x0, y, z};
    double r[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      c[0] = x0 + q;
      r[q] = point_update_space<DIM, LD>(p, keff, un, n, i0 + q, c);
    }
    reinterpret_cast<double2 *>(out + i0)[0] = make_double2(r[0], r[1]);
    reinterpret_cast<double2 *>(out + i0)[1] = make_double2(r[2], r[3]);
    return;
  }
  group_update<DIM, H, LD, AB>(p, keff, un, out, n, x0, y, z);
}

}  // namespace atfd
