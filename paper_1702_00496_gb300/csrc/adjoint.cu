// adjoint.cu -- hand-written adjoint of the AT forward step (gradient of a final-time misfit with respect to
// the initial field and the diffusivity alpha), replaying the recorded delays backward.
//
// Forward step n (fwd.cu) is linear in the stored levels:
//     U^{n+1}_i = s0 U^n_i + sum_a sum_{j != 0} s_{a,j} v_{a,j}(i),
//     v = U^n_{i+j}                                  when i+j lies in i's PE (or the side's delay is 0),
//     v = sum_{m<T} w_m(k) U^{n-k-m}_{i+j}          when i+j is a buffer point of the side with delay k.
// Its transpose sends lambda^{n+1}_i to lambda^n_{i+j} with weight s_{a,j}, or to the older levels
// lambda^{n-k-m}_{i+j} with weight s_{a,j} w_m(k).  The kernel below evaluates that transpose as a GATHER over
// output cells c: each thread owns cells c at every level, so no atomics are needed.  A level l steps back
// receives contributions from backward steps n = l .. l + R - 2, so lambda lives in an R-slot ring (level m in
// slot m mod R): step n reads slot n+1, adds into levels n .. n-R+3, and initialises level n-R+2 (whose slot
// held the consumed lambda^{n+2}).
//
// d/d alpha: s_{a,j} = dt (-c_a cd1_j/dx_a + alpha cd2_j/dx_a^2), so dU^{n+1}_i/d alpha = sum q_{a,j} v_{a,j}(i)
// with q_{a,j} = dt cd2_j / dx_a^2 (the AT second derivative times dt); the kernel accumulates
// <lambda^{n+1}, dt D2_AT U> per block, in a fixed block-to-cell assignment, so the sum is deterministic.
//
// Forward levels for the alpha term come from a segment buffer: the forward pass keeps a checkpoint every s steps
// (s ~ sqrt(steps)); the backward sweep restores one segment at a time, recomputes its levels with the forward
// kernels, and runs the adjoint steps of that segment in reverse.  A checkpoint at step n0 holds U^{n0} in full and,
// of the R-2 older levels the next steps read (Eq. "general_deriv_async": only buffer points are read at delayed
// levels), only the cells within the buffer reach of a PE face -- the strips below.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/at.h"
#include "stencil.cuh"

namespace {

using namespace atfd;

#define AT_MAX_LAG (AT_MAX_L + AT_MAX_T)

struct AdjParams {
  StepParams f;        // forward parameters whose ring is the segment buffer (R = segment depth)
  double *lam;         // adjoint ring, Rl slots of f.ntot
  int32_t Rl;          // = L + T of the problem
  uint8_t *akeff;      // effective delays of the forward steps the backward sweep replays (two buffers)
  double *g_blk;       // per-block accumulators of d J / d alpha
  // grouped shapes: the step kernel's group order (interior groups first, then edge groups: f.order in 3D,
  // group_1d_order in 1D), list_len groups of which the first n_interior are interior
  int64_t list_len, n_interior;
  int32_t alpha;       // accumulate dJ/dalpha (needs the forward levels); 0: lambda only
  // Adams-Bashforth (kernels instantiated with AB): the transposed taps act on mu = sum_m beta_m lambda^{s+1} (the
  // adjoint of dt f^n), and lambda^{n+1} reaches lambda^n through the identity (s0 lacks the 1).
  const double *mu;
  int32_t reach;       // levels a step reaches below n: R - 2 (level n - reach is initialised by step n)
};

// Block sum of v into g_blk[blockIdx.x] (warp shuffles, then warp 0 in warp order).
__device__ __forceinline__ void block_accumulate(double v, double *g_blk) {
  __shared__ double part[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) part[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double s = lane < (int)(blockDim.x >> 5) ? part[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) g_blk[blockIdx.x] += s;
  }
}

// General path for one output cell c (any position): transpose contributions per lag and the alpha term.
template <int DIM, int H, bool AB>
__device__ void adjoint_cell(const AdjParams &a, const uint8_t *__restrict__ keff, int64_t n, int64_t ci,
                             const int c[3], double &galpha) {
  const StepParams &f = a.f;
  const int64_t N = f.ntot;
  const double *lnext = a.lam + ((n + 1) % a.Rl) * N;
  const double *ln = AB ? a.mu : lnext;
  const double *un = f.ring + (n % f.R) * N;
  const int64_t stride[3] = {1, (int64_t)f.n[0], (int64_t)f.n[0] * f.n[1]};
  int pidx[3] = {0, 0, 0}, pos[3] = {0, 0, 0};
#pragma unroll
  for (int ax = 0; ax < DIM; ++ax) {
    pidx[ax] = c[ax] / f.S[ax];
    pos[ax] = c[ax] - pidx[ax] * f.S[ax];
  }
  double acc[AT_MAX_LAG];
#pragma unroll
  for (int l = 0; l < AT_MAX_LAG; ++l) acc[l] = 0.0;
  const double lc = ln[ci];
  acc[0] = fma(f.s0, lc, AB ? lnext[ci] : f.zero);
  double d2 = a.alpha ? fma(f.q0, __ldg(un + ci), f.zero) : 0.0;
#pragma unroll
  for (int ax = 0; ax < DIM; ++ax) {
    const bool edge = f.use_pe[ax] && (pos[ax] < H || pos[ax] >= f.S[ax] - H);
#pragma unroll
    for (int j = -H; j <= H; ++j) {
      if (j == 0) continue;
      // transpose: point i = c - j reads c through its tap j
      const int ia = wrap_coord(c[ax] - j, f.n[ax]);
      const int64_t i = ci + (int64_t)(ia - c[ax]) * stride[ax];
      const double s = f.s[ax][j + H], li = ln[i];
      int k = 0;
      if (edge) {
        const int pi = ia / f.S[ax];
        if (pi != pidx[ax]) {  // c is a buffer point of i, on the side of i's PE that faces c
          int pid[3] = {pidx[0], pidx[1], pidx[2]};
          pid[ax] = pi;
          k = keff[side_of<DIM>(f, pid, ax, j > 0 ? 1 : 0)];
        }
      }
      if (k == 0) {
        acc[0] = fma(s, li, acc[0]);
      } else {
        for (int m = 0; m < f.T; ++m) acc[k + m] = fma(s * f.w[k][m], li, acc[k + m]);
      }
      if (!a.alpha) continue;
      // alpha term: c's own tap j, with c's own side delays
      const int cj = wrap_coord(c[ax] + j, f.n[ax]);
      const int64_t cell = ci + (int64_t)(cj - c[ax]) * stride[ax];
      int kc = 0;
      if (edge && pos[ax] + j < 0) kc = keff[side_of<DIM>(f, pidx, ax, 0)];
      if (edge && pos[ax] + j >= f.S[ax]) kc = keff[side_of<DIM>(f, pidx, ax, 1)];
      const double v = kc > 0 ? halo_value<LdgNC>(f, cell, (int)(n % f.R), kc) : __ldg(un + cell);
      d2 = fma(f.q[ax][j + H], v, d2);
    }
  }
  galpha = fma(lc, d2, galpha);
  const int maxlag = a.reach;
  for (int l = 0; l <= maxlag; ++l) {
    const int64_t level = n - l;
    if (level < 0) break;
    double *slot = a.lam + (level % a.Rl) * N + ci;
    if (l == maxlag) *slot = acc[l];
    else if (l == 0 || acc[l] != 0.0) *slot = *slot + acc[l];
  }
}

// Burgers' equation (1D), one output cell c: the step is U^{n+1}_i = U^n_i + phi_i with phi_i = -U^n_i a1_i + a2_i,
// a1 = dt D1_AT U, a2 = dt alpha D2_AT U (taps b1, b2).  Its transpose, with mu the adjoint of phi (Euler:
// lambda^{n+1}), sends mu_i (b2_j - b1_j U^n_i) from each point i = c - j that reads c through tap j to c's level
// (n, or n-k-m with w_m(k) when c is a buffer point of i), and mu_c (b2_0 - a1_c) plus the identity lambda^{n+1}_c to
// level n.  The alpha term is mu_c dt D2_AT U at c, as for the linear step.  The forward levels are always needed.
template <int H, bool AB>
__device__ void adjoint_cell_burgers(const AdjParams &a, const uint8_t *__restrict__ keff, int64_t n, int64_t ci,
                                     double &galpha) {
  const StepParams &f = a.f;
  const int64_t N = f.ntot;
  const double *lnext = a.lam + ((n + 1) % a.Rl) * N;
  const double *ln = AB ? a.mu : lnext;
  const double *un = f.ring + (n % f.R) * N;
  const int c = (int)ci;
  const int pidx[3] = {c / f.S[0], 0, 0};
  const int pos = c - pidx[0] * f.S[0];
  const int sn = (int)(n % f.R);
  const bool edge = f.use_pe[0] && (pos < H || pos >= f.S[0] - H);
  double acc[AT_MAX_LAG];
#pragma unroll
  for (int l = 0; l < AT_MAX_LAG; ++l) acc[l] = 0.0;
  const double mc = ln[ci], uc = LdgNC::ld(un + ci);
  double a1 = f.zero, d2 = a.alpha ? fma(f.q0, uc, f.zero) : 0.0;
#pragma unroll
  for (int j = -H; j <= H; ++j) {
    if (j == 0) continue;
    // transpose: point i = c - j reads c through its tap j
    const int ia = wrap_coord(c - j, f.n[0]);
    const double li = ln[ia], ui = LdgNC::ld(un + ia);
    const double src = fma(f.b2[j + H], li, -(f.b1[j + H] * li) * ui);
    int k = 0;
    if (edge) {
      const int pi = ia / f.S[0];
      if (pi != pidx[0]) {
        const int pid[3] = {pi, 0, 0};
        k = keff[side_of<1>(f, pid, 0, j > 0 ? 1 : 0)];
      }
    }
    if (k == 0) {
      acc[0] += src;
    } else {
      for (int m = 0; m < f.T; ++m) acc[k + m] = fma(f.w[k][m], src, acc[k + m]);
    }
    // c's own tap j (its first derivative for the direct term, its second for alpha)
    const int cj = wrap_coord(c + j, f.n[0]);
    int kc = 0;
    if (edge && pos + j < 0) kc = keff[side_of<1>(f, pidx, 0, 0)];
    if (edge && pos + j >= f.S[0]) kc = keff[side_of<1>(f, pidx, 0, 1)];
    const double v = kc > 0 ? halo_value<LdgNC>(f, cj, sn, kc) : LdgNC::ld(un + cj);
    a1 = fma(f.b1[j + H], v, a1);
    if (a.alpha) d2 = fma(f.q[0][j + H], v, d2);
  }
  acc[0] += fma(mc, f.b2[H] - a1, lnext[ci]);
  galpha = fma(mc, d2, galpha);
  const int maxlag = a.reach;
  for (int l = 0; l <= maxlag; ++l) {
    const int64_t level = n - l;
    if (level < 0) break;
    double *slot = a.lam + (level % a.Rl) * N + ci;
    if (l == maxlag) *slot = acc[l];
    else if (l == 0 || acc[l] != 0.0) *slot = *slot + acc[l];
  }
}

// Rows expanded in space (order 2, forward Euler), one output cell c.  A point i whose axis-a position is a PE
// edge and whose side there has delay k > 0 takes that axis's edge row: each row tap t with i + j_t = c sends
// ec_t lambda_i to level n (in-PE tap) or n - k (buffer tap).  Every other point reads c through the central taps
// at level n.  c's own centre coefficient leaves out the axes on which c itself takes a row (the row's j = 0 tap
// stands for it).  The alpha term uses the second-derivative part of the same rows (eq) or of the central taps.
template <int DIM>
__device__ void adjoint_cell_space(const AdjParams &a, const uint8_t *__restrict__ keff, int64_t n, int64_t ci,
                                   const int c[3], double &galpha) {
  const StepParams &f = a.f;
  const int64_t N = f.ntot;
  const double *ln = a.lam + ((n + 1) % a.Rl) * N;
  const double *un = f.ring + (n % f.R) * N;
  const int sn = (int)(n % f.R);
  const int64_t stride[3] = {1, (int64_t)f.n[0], (int64_t)f.n[0] * f.n[1]};
  int pidx[3] = {0, 0, 0}, krow[3] = {0, 0, 0}, srow[3] = {0, 0, 0};
#pragma unroll
  for (int ax = 0; ax < DIM; ++ax) pidx[ax] = c[ax] / f.S[ax];
  double c0 = f.ts > 1 ? 0.0 : 1.0;
#pragma unroll
  for (int ax = 0; ax < DIM; ++ax) {
    const int pos = c[ax] - pidx[ax] * f.S[ax];
    if (f.use_pe[ax] && (pos == 0 || pos == f.S[ax] - 1)) {
      srow[ax] = pos == 0 ? 0 : 1;
      krow[ax] = keff[side_of<DIM>(f, pidx, ax, srow[ax])];
    }
    if (krow[ax] == 0) c0 += f.sc[ax];
  }
  double acc[AT_MAX_LAG];
#pragma unroll
  for (int l = 0; l < AT_MAX_LAG; ++l) acc[l] = 0.0;
  const double lc = ln[ci];
  acc[0] = fma(c0, lc, f.zero);
  double d2 = 0.0;
#pragma unroll
  for (int ax = 0; ax < DIM; ++ax) {
    const int jmax = f.use_pe[ax] ? 3 : 1;
    for (int j = -jmax; j <= jmax; ++j) {
      // point i = c - j along axis ax
      const int ia = wrap_coord(c[ax] - j, f.n[ax]);
      const int64_t i = ci + (int64_t)(ia - c[ax]) * stride[ax];
      int ki = 0, si = 0;
      if (f.use_pe[ax]) {
        const int pi = ia / f.S[ax], posi = ia - pi * f.S[ax];
        if (posi == 0 || posi == f.S[ax] - 1) {
          int pid[3] = {pidx[0], pidx[1], pidx[2]};
          pid[ax] = pi;
          si = posi == 0 ? 0 : 1;
          ki = keff[side_of<DIM>(f, pid, ax, si)];
        }
      }
      if (ki > 0) {
        const double li = ln[i];
        for (int t = 0; t < f.ecount[ax][si]; ++t)
          if (f.ej[ax][si][t] == j) {
            const int l = f.ebuf[ax][si][t] ? ki : 0;
            acc[l] = fma(f.ec[ax][si][t], li, acc[l]);
          }
      } else if (j == 1 || j == -1) {
        acc[0] = fma(f.s[ax][j + 1], ln[i], acc[0]);
      }
    }
    if (!a.alpha) continue;
    // c's own second derivative along ax at step n
    if (krow[ax] > 0) {
      const int s = srow[ax];
      for (int t = 0; t < f.ecount[ax][s]; ++t) {
        const int cj = wrap_coord(c[ax] + f.ej[ax][s][t], f.n[ax]);
        const int64_t cell = ci + (int64_t)(cj - c[ax]) * stride[ax];
        const double *lvl = f.ebuf[ax][s][t] ? f.ring + slot_back(sn, krow[ax], f.R) * N : un;
        d2 = fma(f.eq[ax][s][t], LdgNC::ld(lvl + cell), d2);
      }
    } else {
      d2 = fma(f.qc[ax], LdgNC::ld(un + ci), d2);
      for (int j = -1; j <= 1; j += 2) {
        const int cj = wrap_coord(c[ax] + j, f.n[ax]);
        d2 = fma(f.q[ax][j + 1], LdgNC::ld(un + ci + (int64_t)(cj - c[ax]) * stride[ax]), d2);
      }
    }
  }
  galpha = fma(lc, d2, galpha);
  const int maxlag = a.reach;
  for (int l = 0; l <= maxlag; ++l) {
    const int64_t level = n - l;
    if (level < 0) break;
    double *slot = a.lam + (level % a.Rl) * N + ci;
    if (l == maxlag) *slot = acc[l];
    else if (l == 0 || acc[l] != 0.0) *slot = *slot + acc[l];
  }
}

// x taps of the four cells of an edge group: tap j of cell q reads window element t = q + W - j (point i = c - j).
// XT bit 0: the group starts its PE, so the elements t < W lie in the lower x neighbour PE (they read c across
// that PE's upper side) and go to X0; bit 1: the group ends its PE, elements t >= W + 4 lie in the upper one (X1).
// Everything else goes to A.  The buckets are fixed at compile time, so no FMA is issued for a bucket not taken.
template <int H, int XT>
__device__ __forceinline__ void adj_x_taps(const StepParams &f, const double *lv, double A[4], double X0[4],
                                           double X1[4]) {
  constexpr int W = XWin<H>::W;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
#pragma unroll
    for (int j = -H; j <= H; ++j) {
      if (j == 0) continue;
      const int t = q + W - j;
      const double s = f.s[0][j + H];
      if ((XT & 1) && t < W) X0[q] = fma(s, lv[t], X0[q]);
      else if ((XT & 2) && t >= W + 4) X1[q] = fma(s, lv[t], X1[q]);
      else A[q] = fma(s, lv[t], A[q]);
    }
  }
}

// y or z taps of an edge group (3D): points i = c - j along the axis (rows of four cells at stride st).  SIDE 1: the
// row sits at pos = H - CNT, so the taps j > pos (j > H - CNT) reach the lower neighbour PE; SIDE 2: the row sits at
// pos = S - 1 - H + CNT, so the taps j <= pos - S (j < CNT - H) reach the upper one; SIDE 0: every tap stays in the
// PE.  Taps that cross go to X, the others to A.
template <int H, int SIDE, int CNT>
__device__ __forceinline__ void adj_axis_taps(const StepParams &f, int ax, const double *__restrict__ ln, int64_t i0,
                                              int c, int na, int64_t st, double A[4], double X[4]) {
#pragma unroll
  for (int j = -H; j <= H; ++j) {
    if (j == 0) continue;
    const int ia = wrap_coord(c - j, na);
    const int64_t base = i0 + (int64_t)(ia - c) * st;
    const double2 e = LdgNC::ld2(ln + base), g = LdgNC::ld2(ln + base + 2);
    const double lr[4] = {e.x, e.y, g.x, g.y};
    const double s = f.s[ax][j + H];
    const bool cross = (SIDE == 1 && j > H - CNT) || (SIDE == 2 && j < CNT - H);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (cross) X[q] = fma(s, lr[q], X[q]);
      else A[q] = fma(s, lr[q], A[q]);
    }
  }
}

// Case index of an axis position: 0 away from the PE faces, CNT (1..H) for a row CNT cells inside the lower face
// region (pos = H - CNT), H + CNT for CNT cells inside the upper one (pos = S - 1 - H + CNT).
__device__ __forceinline__ int axis_case(const StepParams &f, int ax, int pos, int H) {
  if (!f.use_pe[ax]) return 0;
  if (pos < H) return H - pos;
  if (pos > f.S[ax] - 1 - H) return H + pos - (f.S[ax] - 1 - H);
  return 0;
}

// Side index of the neighbour PE across this PE's lower (or upper) face along axis ax: its upper (lower) side.
template <int DIM>
__device__ __forceinline__ int64_t neighbour_side(const StepParams &f, const int pidx[3], int ax, bool lower) {
  int pid[3] = {pidx[0], pidx[1], pidx[2]};
  pid[ax] = lower ? (pidx[ax] + f.pe[ax] - 1) % f.pe[ax] : (pidx[ax] + 1) % f.pe[ax];
  return side_of<DIM>(f, pid, ax, lower ? 1 : 0);
}

template <int H>
__device__ __forceinline__ void adj_axis_dispatch(const StepParams &f, int ax, int cs, const double *__restrict__ ln,
                                                  int64_t i0, int c, int na, int64_t st, double A[4], double X[4]) {
  switch (cs) {
    case 1: adj_axis_taps<H, 1, 1>(f, ax, ln, i0, c, na, st, A, X); break;
    case 2: if constexpr (H >= 2) adj_axis_taps<H, 1, 2>(f, ax, ln, i0, c, na, st, A, X);
            else adj_axis_taps<H, 2, 1>(f, ax, ln, i0, c, na, st, A, X);
            break;
    case 3: if constexpr (H >= 3) adj_axis_taps<H, 1, 3>(f, ax, ln, i0, c, na, st, A, X);
            else adj_axis_taps<H, 2, 3 - H>(f, ax, ln, i0, c, na, st, A, X);
            break;
    case 4: adj_axis_taps<H, 2, (4 - H > 0 ? 4 - H : 1)>(f, ax, ln, i0, c, na, st, A, X); break;
    case 5: adj_axis_taps<H, 2, (5 - H > 0 ? 5 - H : 1)>(f, ax, ln, i0, c, na, st, A, X); break;
    case 6: adj_axis_taps<H, 2, (6 - H > 0 ? 6 - H : 1)>(f, ax, ln, i0, c, na, st, A, X); break;
    default: adj_axis_taps<H, 0, 0>(f, ax, ln, i0, c, na, st, A, X); break;
  }
}

// Edge group: the four cells x0..x0+3 of row (y, z) when some of them lie within h of a PE edge (or the stencil
// wraps around the domain).  Neighbour points i = c - j in another PE read c as a buffer point; their
// contributions are summed per PE side (one side per axis, two along x) and sent to the levels n-k-m of that
// side's delay k with weights w_m(k) (k = 0: level n itself).  The fresh level n-R+2 is zeroed before any
// contribution lands in it.
template <int DIM, int H, bool AB>
__device__ __forceinline__ void adjoint_group(const AdjParams &a, const uint8_t *__restrict__ keff, int64_t n, int x0,
                                              int y, int z, double &galpha) {
  const StepParams &f = a.f;
  const int64_t N = f.ntot;
  const int nx = f.n[0];
  const int64_t row = DIM == 3 ? ((int64_t)z * f.n[1] + y) * nx : 0;
  const int64_t i0 = row + x0;
  const double *lnext = a.lam + ((n + 1) % a.Rl) * N;
  const double *ln = AB ? a.mu : lnext;
  double d[4] = {0.0, 0.0, 0.0, 0.0};
  double uc[4];
  if (a.alpha) group_eval<DIM, H, LdgNC, true>(f, keff, f.ring + (n % f.R) * N, n, x0, y, z, d, uc);
  int pidx[3] = {x0 / f.S[0], 0, 0}, pos[3] = {0, 0, 0};
  pos[0] = x0 - pidx[0] * f.S[0];
  if (DIM == 3) {
    pidx[1] = y / f.S[1]; pos[1] = y - pidx[1] * f.S[1];
    pidx[2] = z / f.S[2]; pos[2] = z - pidx[2] * f.S[2];
  }
  constexpr int W = XWin<H>::W, NW = XWin<H>::N;
  double lv[NW];
  if (x0 >= W && x0 + 4 + W <= nx) {
#pragma unroll
    for (int t = 0; t < NW; t += 2) {
      const double2 l = LdgNC::ld2(ln + i0 - W + t);
      lv[t] = l.x; lv[t + 1] = l.y;
    }
  } else {
#pragma unroll
    for (int t = 0; t < NW; ++t) lv[t] = LdgNC::ld(ln + row + wrap_coord(x0 - W + t, nx));
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) galpha = fma(lv[q + W], d[q], galpha);
  // x: x0 is a multiple of 4 and h <= 3 < 4, so only a group at the start of its PE (pos 0) reaches the lower
  // PE and only one at its end (pos S-4) the upper; with S = 4 both
  int xt = 0;
  if (f.use_pe[0]) xt = (pos[0] == 0 ? 1 : 0) | (pos[0] + 4 == f.S[0] ? 2 : 0);
  // X[0]: lower x PE, X[1]: upper x PE, X[2]: y neighbour PE, X[3]: z neighbour PE; kX[b] its side's delay, -1 for
  // a bucket this group does not feed
  double A[4], X[4][4];
  int kX[4] = {-1, -1, -1, -1};
  double id[4] = {f.zero, f.zero, f.zero, f.zero};
  if (AB) {
    const double2 e0 = LdgNC::ld2(lnext + i0), e1 = LdgNC::ld2(lnext + i0 + 2);
    id[0] = e0.x; id[1] = e0.y; id[2] = e1.x; id[3] = e1.y;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    A[q] = fma(f.s0, lv[q + W], id[q]);
    X[0][q] = X[1][q] = X[2][q] = X[3][q] = 0.0;
  }
  if (xt & 1) kX[0] = keff[neighbour_side<DIM>(f, pidx, 0, true)];
  if (xt & 2) kX[1] = keff[neighbour_side<DIM>(f, pidx, 0, false)];
  switch (xt) {
    case 1: adj_x_taps<H, 1>(f, lv, A, X[0], X[1]); break;
    case 2: adj_x_taps<H, 2>(f, lv, A, X[0], X[1]); break;
    case 3: adj_x_taps<H, 3>(f, lv, A, X[0], X[1]); break;
    default: adj_x_taps<H, 0>(f, lv, A, X[0], X[1]); break;
  }
  if (DIM == 3) {  // y then z, written out so the buckets stay in registers
    const int cy = axis_case(f, 1, pos[1], H), cz = axis_case(f, 2, pos[2], H);
    if (cy > 0) kX[2] = keff[neighbour_side<DIM>(f, pidx, 1, cy <= H)];
    if (cz > 0) kX[3] = keff[neighbour_side<DIM>(f, pidx, 2, cz <= H)];
    adj_axis_dispatch<H>(f, 1, cy, ln, i0, y, f.n[1], (int64_t)nx, A, X[2]);
    adj_axis_dispatch<H>(f, 2, cz, ln, i0, z, f.n[2], (int64_t)nx * f.n[1], A, X[3]);
  }
  // delay 0: the crossing taps read level n itself
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    if (kX[b] != 0) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) A[q] += X[b][q];
  }
  const int64_t fresh = n - a.reach;
  const int snl = (int)(n % a.Rl);
  double2 *cur = reinterpret_cast<double2 *>(a.lam + snl * N + i0);
  if (a.reach == 0) {
    cur[0] = make_double2(A[0], A[1]);
    cur[1] = make_double2(A[2], A[3]);
    return;
  }
  if (fresh >= 0) {
    double2 *fr = reinterpret_cast<double2 *>(a.lam + slot_back(snl, a.reach, a.Rl) * N + i0);
    fr[0] = make_double2(0.0, 0.0);
    fr[1] = make_double2(0.0, 0.0);
  }
  {
    const double2 p0 = cur[0], p1 = cur[1];
    cur[0] = make_double2(p0.x + A[0], p0.y + A[1]);
    cur[1] = make_double2(p1.x + A[2], p1.y + A[3]);
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int k = kX[b];
    if (k <= 0) continue;
    for (int m = 0; m < f.T; ++m) {
      const double wk = f.w[k][m];
      double2 *o = reinterpret_cast<double2 *>(a.lam + slot_back(snl, k + m, a.Rl) * N + i0);
      const double2 p0 = o[0], p1 = o[1];
      o[0] = make_double2(fma(wk, X[b][0], p0.x), fma(wk, X[b][1], p0.y));
      o[1] = make_double2(fma(wk, X[b][2], p1.x), fma(wk, X[b][3], p1.y));
    }
  }
}

// Backward step n, one launch, which also draws the delays of step n-1.  MODE 0: every cell by the general path
// (shapes without groups of four).  MODE 1: cells in groups of four x points (n[0] % 4 == 0, 16-byte aligned
// slots); a group whose cells and neighbours all lie inside one PE and away from the domain ends takes the
// straight path, the others the edge path (adjoint_group).
#ifndef AT_ADJ_MIN_BLOCKS
#define AT_ADJ_MIN_BLOCKS 3
#endif
template <int MODE>
struct AdjBounds {
  static constexpr int min_blocks = MODE == 1 ? AT_ADJ_MIN_BLOCKS : 2;
};
template <int DIM, int H, int MODE, bool AL, bool AB, bool BG = false, bool SP = false>
__global__ void __launch_bounds__(256, AdjBounds<MODE>::min_blocks) adjoint_step_kernel(const AdjParams a,
                                                                                      const int64_t n) {
  constexpr bool G = MODE != 0;
  const StepParams &f = a.f;
  const int64_t N = f.ntot;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nthreads = (int64_t)gridDim.x * blockDim.x;
  if (n >= 1) draw_sides(f, n - 1, tid, nthreads, a.akeff + ((n - 1) & 1) * f.nb);
  const uint8_t *keff = a.akeff + (n & 1) * f.nb;
  double galpha = 0.0;
  if (!G) {
    const int nx = f.n[0], ny = DIM == 3 ? f.n[1] : 1;
    for (int64_t i = tid; i < N; i += nthreads) {
      int c[3] = {(int)i, 0, 0};
      if (DIM == 3) {
        const int64_t yz = i / nx;
        c[0] = (int)(i - yz * nx); c[2] = (int)(yz / ny); c[1] = (int)(yz - (int64_t)c[2] * ny);
      }
      if constexpr (BG && DIM == 1) adjoint_cell_burgers<H, AB>(a, keff, n, i, galpha);
      else if constexpr (SP) adjoint_cell_space<DIM>(a, keff, n, i, c, galpha);
      else adjoint_cell<DIM, H, AB>(a, keff, n, i, c, galpha);
    }
  } else {
    const double *lnext = a.lam + ((n + 1) % a.Rl) * N;
    const double *ln = AB ? a.mu : lnext;
    const double *un = f.ring + (n % f.R) * N;
    const int nx = f.n[0], ny = f.n[1];
    const int gx = nx >> 2;
    // interior and edge groups in chunks of 32 (one warp, one path): chunk c of C = Ci + Ce is an edge chunk when
    // floor((c+1) Ce / C) > floor(c Ce / C), so edge warps, which wait on memory, spread evenly among interior
    // warps, which keep the FP64 pipe busy
    const int64_t n_edge = a.list_len - a.n_interior;
    const int64_t Ci = (a.n_interior + 31) >> 5, Ce = (n_edge + 31) >> 5, C = Ci + Ce;
    for (int64_t e = tid; e < (C << 5); e += nthreads) {
      const int64_t c = e >> 5, lane = e & 31, ce0 = c * Ce / C;
      const bool edge = (c + 1) * Ce / C > ce0;
      const int64_t k = edge ? a.n_interior + (ce0 << 5) + lane : ((c - ce0) << 5) + lane;
      if (k >= (edge ? a.list_len : a.n_interior)) continue;
      const int64_t g = DIM == 1 ? group_1d_order(f, k) : (int64_t)f.order[k];
      const int64_t r = g / gx;
      const int x0 = (int)(g - r * gx) << 2;
      const int z = DIM == 3 ? (int)(r / ny) : 0, y = DIM == 3 ? (int)(r - (int64_t)z * ny) : 0;
      const int64_t i0 = r * nx + x0;
      if (edge) {
        adjoint_group<DIM, H, AB>(a, keff, n, x0, y, z, galpha);
        continue;
      }
      constexpr int W = XWin<H>::W, NW = XWin<H>::N;
      double lv[NW], uv[NW];
#pragma unroll
      for (int t = 0; t < NW; t += 2) {
        const double2 l = LdgNC::ld2(ln + i0 - W + t);
        lv[t] = l.x; lv[t + 1] = l.y;
        if (AL) {
          const double2 u = LdgNC::ld2(un + i0 - W + t);
          uv[t] = u.x; uv[t + 1] = u.y;
        }
      }
      double A[4], D[4], id[4] = {f.zero, f.zero, f.zero, f.zero};
      if (AB) {
        const double2 e0 = LdgNC::ld2(lnext + i0), e1 = LdgNC::ld2(lnext + i0 + 2);
        id[0] = e0.x; id[1] = e0.y; id[2] = e1.x; id[3] = e1.y;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        double acc = fma(f.s0, lv[q + W], id[q]), d = AL ? fma(f.q0, uv[q + W], f.zero) : 0.0;
#pragma unroll
        for (int j = -H; j <= H; ++j) {
          if (j == 0) continue;
          acc = fma(f.s[0][j + H], lv[q + W - j], acc);
          if (AL) d = fma(f.q[0][j + H], uv[q + W + j], d);
        }
        A[q] = acc;
        D[q] = d;
      }
      if (DIM == 3) {
#pragma unroll
        for (int ax = 1; ax < 3; ++ax) {
          const int64_t st = ax == 1 ? (int64_t)nx : (int64_t)nx * ny;
#pragma unroll
          for (int j = -H; j <= H; ++j) {
            if (j == 0) continue;
            const double2 la = LdgNC::ld2(ln + i0 - j * st), lb = LdgNC::ld2(ln + i0 - j * st + 2);
            double2 ua = make_double2(0.0, 0.0), ub = ua;
            if (AL) { ua = LdgNC::ld2(un + i0 + j * st); ub = LdgNC::ld2(un + i0 + j * st + 2); }
            const double s = f.s[ax][j + H], qq = f.q[ax][j + H];
            A[0] = fma(s, la.x, A[0]); A[1] = fma(s, la.y, A[1]); A[2] = fma(s, lb.x, A[2]); A[3] = fma(s, lb.y, A[3]);
            if (AL) { D[0] = fma(qq, ua.x, D[0]); D[1] = fma(qq, ua.y, D[1]); D[2] = fma(qq, ub.x, D[2]); D[3] = fma(qq, ub.y, D[3]); }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) if (AL) galpha = fma(lv[q + W], D[q], galpha);
      double2 *cur = reinterpret_cast<double2 *>(a.lam + (n % a.Rl) * N + i0);
      if (a.reach == 0) {
        cur[0] = make_double2(A[0], A[1]);
        cur[1] = make_double2(A[2], A[3]);
      } else {
        const double2 p0 = cur[0], p1 = cur[1];
        cur[0] = make_double2(p0.x + A[0], p0.y + A[1]);
        cur[1] = make_double2(p1.x + A[2], p1.y + A[3]);
        const int64_t fresh = n - a.reach;
        if (fresh >= 0) {
          double2 *fr = reinterpret_cast<double2 *>(a.lam + (fresh % a.Rl) * N + i0);
          fr[0] = make_double2(0.0, 0.0);
          fr[1] = make_double2(0.0, 0.0);
        }
      }
    }
  }
  if (AL) block_accumulate(galpha, a.g_blk);
}

// Adams-Bashforth: mu = sum of up to three weighted adjoint levels (the adjoint of dt f^n, see the driver).
struct MuTerms {
  const double *src[3];
  double w[3];
  int32_t count;
};

__global__ void ab_mu_kernel(double *__restrict__ mu, const MuTerms t, int64_t N) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double v = t.w[0] * t.src[0][i];
    for (int k = 1; k < t.count; ++k) v = fma(t.w[k], t.src[k][i], v);
    mu[i] = v;
  }
}

__global__ void sum_blocks_kernel(const double *g_blk, int nblk, double *out) {
  __shared__ double part[32];
  double v = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) v += g_blk[b];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) part[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double s = lane < (int)(blockDim.x >> 5) ? part[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) *out = s;
  }
}

// Cells that any step reads at a delayed level: those within hw cells of a face of their own PE along a split axis
// (a buffer point of a PE lies in the neighbour PE, at most hw cells from the face they share; hw = h for the
// central and time-expanded rows and Burgers' equation, 3 for the rows expanded in space, whose (2,2,2)a row reads
// i-1 .. i-3 across the edge).  They are enumerated without a list, as three disjoint boxes of a mixed-radix index:
//   part Z: z in the strips of z (any y, x);
//   part Y: z outside them, y in the strips of y (any x);
//   part X: z and y outside, x in the strips of x.
// Along an axis, strip coordinate t lies in PE t / w at offset t % w (w = min(2 hw, S) cells per PE: the first hw and
// the last hw cells, or all S when 2 hw >= S); complement coordinate t in PE t / (S - 2 hw), hw cells in.  An axis
// without PE boundaries has no strip cells.
struct StripMap {
  int32_t n[3], S[3], hw[3];
  int64_t cs[3], cc[3];  // strip and complement coordinates per axis
  int64_t part_z, part_y, total;
};

StripMap make_strips(const StepParams &p) {
  StripMap m;
  const int hw = p.scheme >= AT_AT_SPACE2 ? (p.h > 3 ? p.h : 3) : p.h;
  for (int a = 0; a < 3; ++a) {
    m.n[a] = p.n[a];
    m.S[a] = p.S[a];
    const bool split = a < p.dim && p.use_pe[a];
    m.hw[a] = split ? hw : 0;
    const int64_t w = 2 * (int64_t)hw < p.S[a] ? 2 * hw : p.S[a];
    m.cs[a] = split ? (int64_t)p.pe[a] * w : 0;
    m.cc[a] = (int64_t)p.n[a] - m.cs[a];
  }
  m.part_z = m.cs[2] * m.n[1] * m.n[0];
  m.part_y = m.cc[2] * m.cs[1] * m.n[0];
  m.total = m.part_z + m.part_y + m.cc[2] * m.cc[1] * m.cs[0];
  return m;
}

__device__ __forceinline__ int strip_coord(const StripMap &m, int a, int64_t t) {
  const int S = m.S[a], hw = m.hw[a];
  if (2 * hw >= S) return (int)t;  // every cell of the axis
  const int w = 2 * hw;
  const int64_t pe = t / w;
  const int r = (int)(t - pe * w);
  return (int)(pe * S + (r < hw ? r : S - w + r));
}

__device__ __forceinline__ int comp_coord(const StripMap &m, int a, int64_t t) {
  if (m.hw[a] == 0) return (int)t;
  const int w = m.S[a] - 2 * m.hw[a];
  const int64_t pe = t / w;
  return (int)(pe * m.S[a] + m.hw[a] + (t - pe * w));
}

__device__ __forceinline__ int64_t strip_cell(const StripMap &m, int64_t j) {
  const int64_t n0 = m.n[0], n1 = m.n[1];
  int64_t x, y, z;
  if (j < m.part_z) {
    const int64_t row = j / n0;
    x = j - row * n0;
    y = row % n1;
    z = strip_coord(m, 2, row / n1);
  } else if (j - m.part_z < m.part_y) {
    const int64_t k = j - m.part_z, row = k / n0;
    x = k - row * n0;
    y = strip_coord(m, 1, row % m.cs[1]);
    z = comp_coord(m, 2, row / m.cs[1]);
  } else {
    const int64_t k = j - m.part_z - m.part_y, r = k / m.cs[0];
    x = strip_coord(m, 0, k - r * m.cs[0]);
    y = comp_coord(m, 1, r % m.cc[1]);
    z = comp_coord(m, 2, r / m.cc[1]);
  }
  return (z * n1 + y) * n0 + x;
}

// PACK: packed[j] = field[cell(j)]; else field[cell(j)] = packed[j], for j < m.total.
template <bool PACK>
__global__ void strip_copy_kernel(double *__restrict__ field, double *__restrict__ packed, const StripMap m) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m.total; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = strip_cell(m, j);
    if (PACK) packed[j] = field[c];
    else field[c] = packed[j];
  }
}

cudaError_t launch_strip_copy(bool pack, double *field, double *packed, const StripMap &m, cudaStream_t st) {
  if (m.total == 0) return cudaSuccess;
  const int64_t b = (m.total + 255) / 256;
  const int blocks = (int)(b < 152 * 8 ? b : 152 * 8);
  if (pack) strip_copy_kernel<true><<<blocks, 256, 0, st>>>(field, packed, m);
  else strip_copy_kernel<false><<<blocks, 256, 0, st>>>(field, packed, m);
  return cudaGetLastError();
}

const int kAdjThreads = 256;

int adj_blocks() {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms * 8;
}

template <int DIM, int H, bool AL, bool AB>
void launch_modes(const AdjParams &a, int64_t n, int nblk, bool grouped, cudaStream_t st) {
  if constexpr (DIM == 1) {
    if (a.f.burgers) {  // per-cell path
      adjoint_step_kernel<1, H, 0, AL, AB, true><<<nblk, kAdjThreads, 0, st>>>(a, n);
      return;
    }
  }
  if constexpr (H == 1 && !AB) {
    if (a.f.scheme >= AT_AT_SPACE2) {  // rows expanded in space: per-cell path
      adjoint_step_kernel<DIM, 1, 0, AL, false, false, true><<<nblk, kAdjThreads, 0, st>>>(a, n);
      return;
    }
  }
  if (grouped) {
    adjoint_step_kernel<DIM, H, 1, AL, AB><<<nblk, kAdjThreads, 0, st>>>(a, n);
  } else {
    adjoint_step_kernel<DIM, H, 0, AL, AB><<<nblk, kAdjThreads, 0, st>>>(a, n);
  }
}

template <int DIM, int H>
void launch_alpha(const AdjParams &a, int64_t n, int nblk, bool grouped, cudaStream_t st) {
  if (a.mu) {
    if (a.alpha) launch_modes<DIM, H, true, true>(a, n, nblk, grouped, st);
    else launch_modes<DIM, H, false, true>(a, n, nblk, grouped, st);
  } else {
    if (a.alpha) launch_modes<DIM, H, true, false>(a, n, nblk, grouped, st);
    else launch_modes<DIM, H, false, false>(a, n, nblk, grouped, st);
  }
}

bool adjoint_grouped(const AdjParams &a) {
  return a.f.n[0] % 4 == 0 && (!a.f.use_pe[0] || a.f.S[0] % 4 == 0) && (a.f.dim == 1 || a.f.order != nullptr) &&
         (reinterpret_cast<uintptr_t>(a.lam) % 16) == 0 && (reinterpret_cast<uintptr_t>(a.f.ring) % 16) == 0;
}

// The straight (interior) path of the grouped kernel needs a group whose cells and stencil neighbours (the x window of W = h
// rounded up to even cells on each side) lie in its PE and away from the domain ends.  The step kernel's order
// lists exactly those groups first (3D: built at at_init; 1D: group_1d_order, every group of a PE but its first
// and last): with x0 a multiple of 4 and h <= 3, x0 >= h implies x0 >= W and x0 + 3 + h < n implies
// x0 + 3 + W < n, so the two definitions agree.
cudaError_t launch_adjoint_step(const AdjParams &a, int64_t n, int nblk, cudaStream_t st) {
  const bool grouped = adjoint_grouped(a);
  if (a.f.dim == 1) {
    if (a.f.h == 1) launch_alpha<1, 1>(a, n, nblk, grouped, st);
    else if (a.f.h == 2) launch_alpha<1, 2>(a, n, nblk, grouped, st);
    else launch_alpha<1, 3>(a, n, nblk, grouped, st);
  } else {
    if (a.f.h == 1) launch_alpha<3, 1>(a, n, nblk, grouped, st);
    else if (a.f.h == 2) launch_alpha<3, 2>(a, n, nblk, grouped, st);
    else launch_alpha<3, 3>(a, n, nblk, grouped, st);
  }
  return cudaGetLastError();
}

// mu for backward step n of an Adams-Bashforth run started from a caller's field (step s uses l(s) = min(s+1, ts)
// levels): the adjoint of dt f^n is sum over the steps s = n .. n+ts-1 (s < Ns) that use f^n, with m = s - n < l(s),
// of beta^{(l(s))}_m lambda^{s+1}.
cudaError_t launch_ab_mu(const AdjParams &a, const StepParams &p, int64_t n, int64_t Ns, cudaStream_t st) {
  MuTerms t;
  t.count = 0;
  for (int64_t s = n; s < n + p.ts && s < Ns; ++s) {
    const int64_t m = s - n;
    const int l = (int)(s + 1 < p.ts ? s + 1 : p.ts);
    if (m >= l) continue;
    t.src[t.count] = a.lam + ((s + 1) % a.Rl) * p.ntot;
    t.w[t.count] = p.beta[l - 1][m];
    ++t.count;
  }
  const int64_t b = (p.ntot + 255) / 256;
  ab_mu_kernel<<<(int)(b < 152 * 16 ? b : 152 * 16), 256, 0, st>>>(const_cast<double *>(a.mu), t, p.ntot);
  return cudaGetLastError();
}

int fail(int code, const char *msg) {
  at_internal_set_error(msg);
  return code;
}

int cuda_fail(cudaError_t e, const char *where) {
  char buf[200];
  std::snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  at_internal_set_error(buf);
  return AT_ERR_CUDA;
}

}  // namespace

namespace {

// Workspace layout (doubles, each part rounded up to 32 doubles):
//   checkpoints  nck x ck_len             for every checkpoint n0 = 0, s, 2s, ...: U^{n0} (ntot), the strip cells of
//                                         levels n0-R+2 .. n0-1 ((R-2) x nstrip), the ts-1 stored right-hand sides
//   segment      (s + R - 1) x ntot       levels of the segment being replayed (level m in slot m mod depth)
//   segment rhs  (ts - 1) x ntot          its stored right-hand sides (Adams-Bashforth)
//   lambda       (R + ts - 1) x ntot      adjoint ring
//   mu           ntot                     Adams-Bashforth: the adjoint of dt f^n
//   g_blk        nblk                     per-block d J / d alpha accumulators, then the sum
//   delays       2 x 2 x nb bytes         effective delays of the recompute and of the backward sweep
struct AdjLayout {
  int64_t s, nck, seg_depth, lam_slots, ck, seg, segf, lam, mu, gblk, keff, total;
  int64_t nstrip, ck_len, ck_strips, ck_rhs;  // strip cells; one checkpoint's length and the offsets of its parts
};

int64_t up32(int64_t v) { return (v + 31) / 32 * 32; }

AdjLayout layout(const at_handle *hd, int64_t nsteps, int64_t every) {
  AdjLayout L;
  const int64_t N = hd->sp.ntot, R = hd->sp.R;
  L.s = every > 0 ? every : (int64_t)std::ceil(std::sqrt((double)(nsteps > 0 ? nsteps : 1)));
  if (L.s < 1) L.s = 1;
  L.nck = nsteps > 0 ? (nsteps + L.s - 1) / L.s : 0;
  const int64_t nf = hd->sp.ts - 1;  // Adams-Bashforth: stored right-hand sides, part of the forward state
  L.seg_depth = L.s + R - 1;
  L.nstrip = make_strips(hd->sp).total;
  L.ck_strips = up32(N);
  L.ck_rhs = L.ck_strips + up32((R > 2 ? R - 2 : 0) * L.nstrip);
  L.ck_len = L.ck_rhs + nf * up32(N);
  L.lam_slots = R + nf;             // the adjoint levels n+1+m that mu still needs stay alive
  L.ck = 0;
  L.seg = L.ck + L.nck * L.ck_len;
  L.segf = L.seg + up32(L.seg_depth * N);
  L.lam = L.segf + up32(nf * N);
  L.mu = L.lam + up32(L.lam_slots * N);
  L.gblk = L.mu + up32(nf > 0 ? N : 0);
  L.keff = L.gblk + up32(adj_blocks() + 1);
  L.total = L.keff + up32((4 * hd->sp.nb + 7) / 8);
  return L;
}

cudaError_t copy_field(double *dst, const double *src, int64_t n, cudaStream_t st) {
  return cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, st);
}

}  // namespace

// The transposed step covers every scheme (central, time-expanded and space-expanded rows), orders 2, 4 and 6,
// forward Euler and Adams-Bashforth runs started from a caller's field, the linear and Burgers' equations.
static int adjoint_supported(const at_handle *hd) {
  if (hd->sp.ts > 1 && hd->ab_analytic)
    return fail(AT_ERR_STATE, "adjoint: an Adams-Bashforth run must start from a caller's field (at_reset with "
                              "u0_dev): the analytic pre-history depends on alpha");
  return AT_OK;
}

extern "C" int at_adjoint_workspace(at_handle_t *hd, int64_t nsteps, int64_t ckpt_every, int64_t *work_len) {
  if (!hd || nsteps < 0 || ckpt_every < 0 || !work_len) return fail(AT_ERR_ARG, "at_adjoint_workspace: bad argument");
  if (int rc = adjoint_supported(hd)) return rc;
  *work_len = layout(hd, nsteps, ckpt_every).total;
  return AT_OK;
}

extern "C" int at_adjoint_forward(at_handle_t *hd, int64_t nsteps, int64_t ckpt_every, double *work_dev,
                                  int64_t work_len) {
  if (!hd || nsteps < 0 || ckpt_every < 0 || !work_dev) return fail(AT_ERR_ARG, "at_adjoint_forward: bad argument");
  if (int rc = adjoint_supported(hd)) return rc;
  if (hd->step != 0) return fail(AT_ERR_STATE, "at_adjoint_forward: the handle must be at step 0 (at_reset)");
  const AdjLayout L = layout(hd, nsteps, ckpt_every);
  if (work_len < L.total) return fail(AT_ERR_ARG, "at_adjoint_forward: workspace too small");
  if (reinterpret_cast<uintptr_t>(work_dev) % 16) return fail(AT_ERR_ARG, "at_adjoint_forward: workspace not 16-byte aligned");
  // at_step's limits, checked before any step so a refused pass leaves the handle at step 0
  if (hd->sp.log && nsteps > hd->log_steps) return fail(AT_ERR_STATE, "at_adjoint_forward: delay log is full");
  if (nsteps > 0xFFFFFFFFll) return fail(AT_ERR_STATE, "at_adjoint_forward: step counter exceeds 32 bits");
  const int64_t N = hd->sp.ntot, R = hd->sp.R;
  hd->adj_nsteps = -1;
  hd->adj_resident = false;
  if (L.nck == 1 && nsteps > 0) {
    // One segment covers the whole run: step it inside the segment buffer, which then holds every level the
    // backward sweep needs, so the sweep recomputes nothing.  The handle's ring gets the last live levels.
    cudaStream_t st = hd->stream;
    StepParams seg = hd->sp;
    seg.ring = work_dev + L.seg;
    seg.R = (int32_t)L.seg_depth;
    seg.frhs = hd->sp.ts > 1 ? work_dev + L.segf : nullptr;
    seg.keff = reinterpret_cast<uint8_t *>(work_dev + L.keff);
    cudaError_t e = copy_field(seg.ring, hd->sp.ring, N, st);  // level 0
    for (int64_t m = 0; m + 1 < hd->sp.ts && e == cudaSuccess; ++m)
      e = copy_field(seg.frhs + m * N, hd->sp.frhs + m * N, N, st);
    if (e == cudaSuccess) e = launch_draw_delays(seg, 0, st);
    for (int64_t n = 0; n < nsteps && e == cudaSuccess; ++n) e = launch_forward_step(seg, n, nullptr, st);
    for (int64_t lev = nsteps - R + 2; lev <= nsteps && e == cudaSuccess; ++lev)
      if (lev >= 0) e = copy_field(hd->sp.ring + (lev % R) * N, seg.ring + (lev % seg.R) * N, N, st);
    for (int64_t m = 0; m + 1 < hd->sp.ts && e == cudaSuccess; ++m)
      e = copy_field(hd->sp.frhs + m * N, seg.frhs + m * N, N, st);
    if (e == cudaSuccess) e = launch_draw_delays(hd->sp, nsteps, st);  // as at_step leaves them
    if (e != cudaSuccess) return cuda_fail(e, "at_adjoint_forward");
    hd->step = nsteps;
    hd->adj_resident = true;
  }
  const StripMap strips = make_strips(hd->sp);
  for (int64_t c = 0; !hd->adj_resident && c < L.nck; ++c) {
    const int64_t n0 = c * L.s;
    double *ck = work_dev + L.ck + c * L.ck_len;
    cudaError_t e = copy_field(ck, hd->sp.ring + (n0 % R) * N, N, hd->stream);  // U^{n0} in full
    for (int64_t lev = n0 - R + 2; lev < n0 && e == cudaSuccess; ++lev)  // older levels: the strip cells only
      if (lev >= 0)
        e = launch_strip_copy(true, hd->sp.ring + (lev % R) * N, ck + L.ck_strips + (lev - (n0 - R + 2)) * L.nstrip,
                              strips, hd->stream);
    for (int64_t m = 0; m + 1 < hd->sp.ts && e == cudaSuccess; ++m)  // the stored right-hand sides, slot by slot
      e = copy_field(ck + L.ck_rhs + m * up32(N), hd->sp.frhs + m * N, N, hd->stream);
    if (e != cudaSuccess) return cuda_fail(e, "at_adjoint_forward: checkpoint");
    // single steps (no K-step blocks): the recompute of the backward sweep repeats exactly these launches
    const int64_t todo = (n0 + L.s <= nsteps) ? L.s : nsteps - n0;
    for (int64_t t = 0; t < todo; ++t) {
      cudaError_t e = launch_forward_step(hd->sp, hd->step, nullptr, hd->stream);
      if (e != cudaSuccess) return cuda_fail(e, "at_adjoint_forward: step");
      hd->step += 1;
    }
  }
  hd->adj_nsteps = nsteps;
  hd->adj_every = L.s;
  hd->adj_work = work_dev;
  hd->adj_work_len = work_len;
  return AT_OK;
}

extern "C" int at_adjoint_backward(at_handle_t *hd, const double *lambda_dev, double *grad_u0_dev,
                                   double *grad_alpha_host) {
  if (!hd || !lambda_dev || !grad_u0_dev) return fail(AT_ERR_ARG, "at_adjoint_backward: bad argument");
  if (int rc = adjoint_supported(hd)) return rc;
  const bool want_alpha = grad_alpha_host != nullptr;
  if (hd->adj_nsteps < 0 || hd->step != hd->adj_nsteps)
    return fail(AT_ERR_STATE, "at_adjoint_backward: needs the at_adjoint_forward pass right before");
  const int64_t Ns = hd->adj_nsteps, N = hd->sp.ntot, R = hd->sp.R;
  const AdjLayout L = layout(hd, Ns, hd->adj_every);
  double *w = hd->adj_work;
  cudaStream_t st = hd->stream;
  cudaError_t e = cudaSuccess;
  const int nblk = adj_blocks();
  const StripMap strips = make_strips(hd->sp);
  // segment parameters: forward levels in the segment buffer, no log, own delay buffers
  StepParams seg = hd->sp;
  seg.ring = w + L.seg;
  seg.R = (int32_t)L.seg_depth;
  seg.frhs = hd->sp.ts > 1 ? w + L.segf : nullptr;
  seg.log = nullptr;
  seg.log_steps = 0;
  seg.keff = reinterpret_cast<uint8_t *>(w + L.keff);
  AdjParams a;
  a.f = seg;
  a.lam = w + L.lam;
  a.Rl = (int32_t)L.lam_slots;
  a.reach = (int32_t)(R - 2);
  a.mu = hd->sp.ts > 1 ? w + L.mu : nullptr;
  const int64_t Rl = a.Rl;
  a.akeff = reinterpret_cast<uint8_t *>(w + L.keff) + 2 * hd->sp.nb;
  a.g_blk = w + L.gblk;
  a.alpha = want_alpha ? 1 : 0;
  // the linear transposed step needs the forward levels only for the alpha term; Burgers' always does
  const bool need_fwd = (want_alpha || hd->sp.burgers) && !hd->adj_resident;  // resident: levels are in place
  // grouped shapes: the step kernel's group order, interior groups at its head
  a.list_len = 0;
  a.n_interior = 0;
  if (adjoint_grouped(a)) {
    a.list_len = N / 4;
    if (hd->sp.dim == 3) {
      a.n_interior = hd->n_interior;
    } else {  // group_1d_order: the groups between the first and the last of each PE, PE by PE
      const int64_t gS = (hd->sp.use_pe[0] ? hd->sp.S[0] : hd->sp.n[0]) / 4;
      a.n_interior = gS < 3 ? 0 : (hd->sp.n[0] / 4 / gS) * (gS - 2);
    }
  }
  // lambda^Ns = the caller's seed; the R-2 older levels start at zero; alpha accumulators at zero
  e = copy_field(a.lam + (Ns % Rl) * N, lambda_dev, N, st);
  for (int64_t m = 1; m <= R - 2 && e == cudaSuccess; ++m)
    if (Ns - m >= 0) e = cudaMemsetAsync(a.lam + ((Ns - m) % Rl) * N, 0, sizeof(double) * (size_t)N, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.g_blk, 0, sizeof(double) * (size_t)(nblk + 1), st);
  if (e == cudaSuccess && Ns > 0) {
    StepParams first = seg;
    first.keff = a.akeff;
    e = launch_draw_delays(first, Ns - 1, st);
  }
  for (int64_t c = L.nck - 1; c >= 0 && e == cudaSuccess; --c) {
    const int64_t n0 = c * L.s, n1 = (n0 + L.s < Ns) ? n0 + L.s : Ns;
    double *ck = w + L.ck + c * L.ck_len;
    if (need_fwd) e = copy_field(seg.ring + (n0 % seg.R) * N, ck, N, st);
    for (int64_t lev = n0 - R + 2; need_fwd && lev < n0 && e == cudaSuccess; ++lev)
      if (lev >= 0)
        e = launch_strip_copy(false, seg.ring + (lev % seg.R) * N, ck + L.ck_strips + (lev - (n0 - R + 2)) * L.nstrip,
                              strips, st);
    for (int64_t m = 0; need_fwd && m + 1 < hd->sp.ts && e == cudaSuccess; ++m)
      e = copy_field(seg.frhs + m * N, ck + L.ck_rhs + m * up32(N), N, st);
    // the forward levels serve the alpha term (and Burgers' transposed step): without them no recompute
    if (need_fwd && e == cudaSuccess) e = launch_draw_delays(seg, n0, st);
    for (int64_t n = n0; need_fwd && n + 1 < n1 && e == cudaSuccess; ++n) e = launch_forward_step(seg, n, nullptr, st);
    for (int64_t n = n1 - 1; n >= n0 && e == cudaSuccess; --n) {
      if (a.mu) e = launch_ab_mu(a, hd->sp, n, Ns, st);
      if (e == cudaSuccess) e = launch_adjoint_step(a, n, nblk, st);
    }
  }
  if (e == cudaSuccess) e = copy_field(grad_u0_dev, a.lam, N, st);  // level 0 lives in slot 0
  if (want_alpha && e == cudaSuccess) {
    sum_blocks_kernel<<<1, 256, 0, st>>>(a.g_blk, nblk, a.g_blk + nblk);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(grad_alpha_host, a.g_blk + nblk, sizeof(double), cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "at_adjoint_backward");
  if (want_alpha && !std::isfinite(*grad_alpha_host)) return fail(AT_ERR_NONFINITE, "at_adjoint_backward: non-finite gradient");
  return AT_OK;
}
