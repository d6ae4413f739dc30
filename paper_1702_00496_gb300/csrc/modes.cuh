// modes.cuh -- the sum over the initial-condition modes of one axis (Eq. "IC"; Eq. "ana_sol" at time t), shared by
// the single-problem kernels (wave.cu) and the ensemble engine (ensemble.cu), so both produce the same bits.
#pragma once
#include "internal.h"

namespace atfd {

// sum_q A_q sin(k_q x + phi'_q) at x = pi xpi (grid point i of n: xpi = i (2 / n), exact for n a power of two),
// each mode adding ac sin kx + as cos kx (two FMAs), from one sincospi and, over the wavenumbers k = 2 .. kmax,
//   kmax <= 16: the three-term recurrences sin (k+1)x = 2 cos x sin kx - sin (k-1)x (and the same for cos), one
//               FMA each per wavenumber.  A rounding error made at wavenumber j reaches k multiplied by
//               sin((k-j)x)/sin x, at most k - j in size: under kmax^2/2 ulp in all, 1.4e-14 at kmax = 16;
//   kmax > 16:  the rotation (cos kx, sin kx) = (cos (k-1)x, sin (k-1)x) x (cos x, sin x), two multiplies and two
//               FMAs per wavenumber, whose errors add up linearly (a few ulp per rotation).
// Requires ms.rot.
__device__ __forceinline__ double mode_sum(const ModeSet &ms, int nmodes, double xpi) {
  double sx, cx;
  sincospi(xpi, &sx, &cx);
  double sk = sx, ck = cx, s = 0.0;
  int q = 0;
  if (ms.kmax <= 16) {
    const double tc = cx + cx;
    double sp = 0.0, cp = 1.0;  // sin, cos of (k-1)x
    for (int k = 1; k <= ms.kmax; ++k) {
      if (k > 1) {
        const double ns = fma(tc, sk, -sp), nc = fma(tc, ck, -cp);
        sp = sk; cp = ck;
        sk = ns; ck = nc;
      }
      while (q < nmodes && ms.kr[q] == k) {
        s = fma(ms.as[q], ck, fma(ms.ac[q], sk, s));
        ++q;
      }
    }
    return s;
  }
  for (int k = 1; k <= ms.kmax; ++k) {
    if (k > 1) {
      const double ns = fma(sk, cx, ck * sx), nc = fma(ck, cx, -(sk * sx));
      sk = ns;
      ck = nc;
    }
    while (q < nmodes && ms.kr[q] == k) {
      s = fma(ms.as[q], ck, fma(ms.ac[q], sk, s));
      ++q;
    }
  }
  return s;
}

}  // namespace atfd
