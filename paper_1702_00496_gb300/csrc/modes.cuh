// modes.cuh -- the sum over the initial-condition modes of one axis (Eq. "IC"; Eq. "ana_sol" at time t), shared by
// the single-problem kernels (wave.cu) and the ensemble engine (ensemble.cu), so both produce the same bits.
#pragma once
#include "internal.h"

namespace atfd {

// sum_q A_q sin(k_q x + phi'_q) from one sincos of x and the rotation recurrence
//   (cos kx, sin kx) = (cos (k-1)x, sin (k-1)x) x (cos x, sin x),
// each mode adding ac sin kx + as cos kx: two FMAs per mode and four per wavenumber instead of a sine per mode
// (the error grows by a few ulp per rotation).  Requires ms.rot.
__device__ __forceinline__ double mode_sum(const ModeSet &ms, int nmodes, double x) {
  double sx, cx;
  sincos(x, &sx, &cx);
  double sk = sx, ck = cx, s = 0.0;
  int q = 0;
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
