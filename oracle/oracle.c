/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the asynchrony-tolerant (AT) finite-difference
 * method of Aditya & Donzis, "High-order asynchrony-tolerant finite difference schemes for
 * partial differential equations" (arXiv:1702.00496).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference legs may load or call this library.  It shares no code, header, table or constant
 * generator with the CUDA path (paper_1702_00496_gb300/); the two are compared on the same seeded
 * inputs, which the caller passes in (initial-condition amplitudes, phases, wavenumbers, delay
 * thresholds).
 *
 * What it computes, in the paper's own terms:
 *   - grid and PE decomposition: Sec. 2 (Fig. "grid"); periodic domain [0, 2pi): Sec. 5.1.
 *   - delay process: Sec. 5.1 "simulate delays" -- one uniform draw per PE side per step, binned
 *     by {p_0..p_{L-1}}.  The uniform draw is a Philox4x32-10 word (Salmon et al., SC'11), keyed by
 *     the seed and counted by (step, side), so any delay can be replayed.
 *   - spatial operators: the central differences and the AT stencils exactly as printed in the
 *     tables "atschemes-left" / "atschemes-right" ((1,2,2)b, (2,2,2)b, (1,4,2), (2,4,2), (2,6,2), and the
 *     stencils expanded in space, (1,2,2)a, (2,2,2)a, (2,1,2)), written out as the explicit sum over
 *     (point, time level) pairs of Eq. "general_deriv_at2".
 *     ASYNC_STD is the standard scheme read at delayed levels, Eq. "general_deriv_async".
 *   - time integration: forward Euler (one level of Eq. "time_disc"), or Adams-Bashforth with two (Eq.
 *     "time_ab2") or three levels, started with Euler and then AB2.
 *   - the viscous Burgers' equation (Sec. 5.1: Eq. "general" with beta_1 = u, beta_2 = alpha; Case 6):
 *     f = -U_i^n D1 U + alpha D2 U with the same AT D1 and D2, U_i^n the point's own (current) value.
 *   - error: E = U - u_a (Sec. 5.1, Eq. "ana_sol", with the travelling phase read as
 *     sin(kappa (x - c t) + phi)); averages over I, I_I and I_B (Sec. 4).
 *   - adjoint: the literal transpose of the forward step over the stored history (Burgers' equation: the
 *     D1 taps carry -U_i^n and U_i^n itself receives -D1 U, the derivative of the nonlinear term).
 *
 * Readings where the paper is silent:
 *   - a PE side uses one delay for all its buffer points (uniform delay, Sec. 5.1); the two sides
 *     of a shared face are different messages and draw independently;
 *   - levels before 0 do not exist: a drawn delay k>0 is clamped to min(k, max(0, n-(T-1)));
 *   - for the 4th-order point one cell in from a PE edge only the outer stencil point is a
 *     buffer point, so only it is read at delayed levels (Eq. "general_deriv_async");
 *   - an axis split into a single PE has no PE boundary (its periodic wrap is local);
 *   - like every AT row, the stencils expanded in space (Cases 2 and 3) replace the central difference only
 *     when the side's delay is k > 0: they do not reduce to it at k = 0, and used there they leave a jump
 *     across the PE boundary undamped (both edge rows vanish on a step), which makes the synchronous run
 *     first-order accurate, against the slope -2 Sec. 5.2 reports for p_0 = 1;
 *   - (1,2,2)a at the left boundary is read with +U_{i-1}^{n-k}: the printed minus sign makes the row
 *     inconsistent (its coefficients would not sum to zero), and the plus sign gives the mirror image of the
 *     right-boundary row and of Example 1's uniform-delay scheme (Eq. "ex1-1").
 *
 * Compiled with -ffp-contract=off so every product and sum rounds as written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_SYNC 0
#define ORC_ASYNC_STD 1
#define ORC_AT 2
#define ORC_AT_SPACE2 3 /* Case 3: (1,2,2)a and (2,2,2)a at PE edges (order 2) */
#define ORC_AT_SPACE1 4 /* Case 2: (2,1,2) at PE edges (order 2, diffusion only) */

typedef struct {
  int32_t dim;      /* 1 or 3 */
  int32_t order;    /* 2 or 4 */
  int32_t L;        /* delays take values 0..L-1 */
  int32_t scheme;   /* ORC_SYNC, ORC_ASYNC_STD, ORC_AT, ORC_AT_SPACE2, ORC_AT_SPACE1 */
  int64_t n[3];     /* points per axis; unused axes hold 1 */
  int32_t pe[3];    /* PEs per axis; unused axes hold 1 */
  int32_t nmodes;   /* initial-condition modes per axis */
  double c[3];      /* advection speed per axis */
  double alpha;     /* diffusivity */
  double dt;        /* time step */
  uint64_t seed;    /* Philox key */
  const uint64_t *thresholds; /* L-1 ascending cumulative thresholds in [0, 2^32], or NULL: uniform */
  const double *amp;          /* [dim][nmodes] */
  const double *phase;        /* [dim][nmodes] */
  const int32_t *kappa;       /* [dim][nmodes] */
  int32_t tsteps;             /* time integration: 0 or 1 forward Euler, 2 AB2, 3 AB3 (Eq. "time_disc") */
  int32_t burgers;            /* 1: the viscous Burgers' equation u_t + u u_x = alpha u_xx (Sec. 5.1, beta_1 = u,
                                 beta_2 = alpha; Case 6), 1D with c = 0 */
} orc_cfg;

typedef struct {
  int32_t j; /* spatial offset of the stencil point */
  int32_t l; /* time lag: the point is read at level n - l */
  double c;  /* coefficient, already divided by dx^d */
} orc_tap;

static int g_threads = 1;
void orc_set_threads(int t) { g_threads = t < 1 ? 1 : t; }
int orc_have_openmp(void) {
#ifdef _OPENMP
  return 1;
#else
  return 0;
#endif
}

/* ---------------------------------------------------------------- Philox4x32-10 (SC'11) */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Sec. 5.1: a uniform draw on [0,1) -- here the 32-bit word x0 / 2^32 -- falls in one of L bins of
 * widths p_0..p_{L-1}; the bin index is the delay.  Uniform bins: k = floor(x0 * L / 2^32).
 * Given bins: k = number of cumulative thresholds t_m <= x0. */
int orc_delay_raw(uint64_t seed, int64_t step, int64_t side, int L, const uint64_t *thr) {
  uint32_t ctr[4] = {(uint32_t)step, (uint32_t)side, 0u, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t x[4];
  orc_philox4x32_10(ctr, key, x);
  if (thr == NULL) return (int)(((uint64_t)x[0] * (uint64_t)L) >> 32);
  int k = 0;
  for (int m = 0; m < L - 1; ++m)
    if ((uint64_t)x[0] >= thr[m]) k += 1;
  return k;
}

/* number of successive delayed levels a scheme reads at a buffer point */
int orc_time_width(int order, int scheme) { return scheme == ORC_AT ? order / 2 + 1 : 1; }
/* the stencils expanded in space read one delayed level (T = 1) */

/* levels before 0 do not exist: clamp a drawn delay so that level n-k-(T-1) >= 0 */
int orc_delay_effective(int k, int64_t n, int T) {
  if (k <= 0) return 0;
  int64_t lim = n - (T - 1);
  if (lim < 0) lim = 0;
  return (int64_t)k < lim ? k : (int)lim;
}

/* ------------------------------------------------------------------ stencils (tables) */
/* Standard central differences, numerator weights for j = -h..h and the common denominator,
 * as they appear inside the AT table rows:
 *   CD2, d=1: (U_{i+1} - U_{i-1}) / (2 dx)
 *   CD2, d=2: (U_{i+1} - 2 U_i + U_{i-1}) / dx^2
 *   CD4, d=1: (-U_{i+2} + 8 U_{i+1} - 8 U_{i-1} + U_{i-2}) / (12 dx)
 *   CD4, d=2: (-U_{i+2} + 16 U_{i+1} - 30 U_i + 16 U_{i-1} - U_{i-2}) / (12 dx^2)
 *   CD6, d=2: (2 U_{i+3} - 27 U_{i+2} + 270 U_{i+1} - 490 U_i + 270 U_{i-1} - 27 U_{i-2} + 2 U_{i-3}) / (180 dx^2)
 *   CD6, d=1: (U_{i+3} - 9 U_{i+2} + 45 U_{i+1} - 45 U_{i-1} + 9 U_{i-2} - U_{i-3}) / (60 dx), the textbook sixth-
 *             order first derivative (the paper's sixth-order case is pure diffusion and prints none)      */
static const double CD2_D1[3] = {-1.0, 0.0, 1.0};
static const double CD2_D2[3] = {1.0, -2.0, 1.0};
static const double CD4_D1[5] = {1.0, -8.0, 0.0, 8.0, -1.0};
static const double CD4_D2[5] = {-1.0, 16.0, -30.0, 16.0, -1.0};
static const double CD6_D1[7] = {-1.0, 9.0, -45.0, 0.0, 45.0, -9.0, 1.0};
static const double CD6_D2[7] = {2.0, -27.0, 270.0, -490.0, 270.0, -27.0, 2.0};

static void cd_table(int order, int deriv, const double **num, double *den) {
  if (order == 2) {
    *num = deriv == 1 ? CD2_D1 : CD2_D2;
    *den = deriv == 1 ? 2.0 : 1.0;
  } else if (order == 4) {
    *num = deriv == 1 ? CD4_D1 : CD4_D2;
    *den = 12.0;
  } else {
    *num = deriv == 1 ? CD6_D1 : CD6_D2;
    *den = deriv == 1 ? 60.0 : 180.0;
  }
}

/* Weights of the delayed copies in the (1,4,2) and (2,4,2) rows:
 *   (1/2)(k^2+3k+2) at level n-k, -(k^2+2k) at n-k-1, (1/2)(k^2+k) at n-k-2. */
static void w_order4(int k, double w[3]) {
  double kk = (double)k;
  w[0] = 0.5 * (kk * kk + 3.0 * kk + 2.0);
  w[1] = -(kk * kk + 2.0 * kk);
  w[2] = 0.5 * (kk * kk + kk);
}

/* Weights of the delayed copies in the (2,6,2) rows (read with U_{i-3} where the left rows print U_{i+3}):
 *   (1/6)(k^3+6k^2+11k+6), -(1/2)(k^3+5k^2+6k), (1/2)(k^3+4k^2+3k), -(1/6)(k^3+3k^2+2k)
 * at levels n-k, n-k-1, n-k-2, n-k-3. */
static void w_order6(int k, double w[4]) {
  double kk = (double)k, k2 = kk * kk, k3 = k2 * kk;
  w[0] = (k3 + 6.0 * k2 + 11.0 * kk + 6.0) / 6.0;
  w[1] = -(k3 + 5.0 * k2 + 6.0 * kk) / 2.0;
  w[2] = (k3 + 4.0 * k2 + 3.0 * kk) / 2.0;
  w[3] = -(k3 + 3.0 * k2 + 2.0 * kk) / 6.0;
}

static double dxpow(double dx, int d) { return d == 1 ? dx : dx * dx; }

/* The AT stencils expanded in space (tables "atschemes-left/right"), at the PE-edge point of a second-order
 * scheme; buffer points read at level n-k.  dxd = dx^d.  Returns the number of taps.
 *   (1,2,2)a left : (3 U_{i+1} - 3 U_i + U_{i-1}^{n-k} - U_{i-2}^{n-k}) / (4 dx)          (sign of U_{i-1}: see top)
 *   (1,2,2)a right: (U_{i+2}^{n-k} - U_{i+1}^{n-k} + 3 U_i - 3 U_{i-1}) / (4 dx)
 *   (2,2,2)a left : (2 U_{i+2} - 4 U_{i+1} + 2 U_i + U_{i-1}^{n-k} - 2 U_{i-2}^{n-k} + U_{i-3}^{n-k}) / (3 dx^2)
 *   (2,2,2)a right: (U_{i+3}^{n-k} - 2 U_{i+2}^{n-k} + U_{i+1}^{n-k} + 2 U_i - 4 U_{i-1} + 2 U_{i-2}) / (3 dx^2)
 *   (2,1,2)  left : (U_{i+1} - U_i - U_{i-1}^{n-k} + U_{i-2}^{n-k}) / (2 dx^2)
 *   (2,1,2)  right: (U_{i+2}^{n-k} - U_{i+1}^{n-k} - U_i + U_{i-1}) / (2 dx^2)
 * The (2,1,2) rows give only a second derivative; a first derivative is not defined for that case (diffusion).
 * Called for k > 0 only. */
static int space_expanded_taps(int scheme, int deriv, int left, int k, double dxd, orc_tap *out) {
  static const int A1L_j[4] = {1, 0, -1, -2}, A1L_d[4] = {0, 0, 1, 1};
  static const double A1L_c[4] = {3.0, -3.0, 1.0, -1.0};
  static const int A1R_j[4] = {2, 1, 0, -1}, A1R_d[4] = {1, 1, 0, 0};
  static const double A1R_c[4] = {1.0, -1.0, 3.0, -3.0};
  static const int A2L_j[6] = {2, 1, 0, -1, -2, -3}, A2L_d[6] = {0, 0, 0, 1, 1, 1};
  static const double A2L_c[6] = {2.0, -4.0, 2.0, 1.0, -2.0, 1.0};
  static const int A2R_j[6] = {3, 2, 1, 0, -1, -2}, A2R_d[6] = {1, 1, 1, 0, 0, 0};
  static const double A2R_c[6] = {1.0, -2.0, 1.0, 2.0, -4.0, 2.0};
  static const int S2L_j[4] = {1, 0, -1, -2}, S2L_d[4] = {0, 0, 1, 1};
  static const double S2L_c[4] = {1.0, -1.0, -1.0, 1.0};
  static const int S2R_j[4] = {2, 1, 0, -1}, S2R_d[4] = {1, 1, 0, 0};
  static const double S2R_c[4] = {1.0, -1.0, -1.0, 1.0};
  const int *js, *ds;
  const double *cs;
  int nt;
  double den;
  if (scheme == ORC_AT_SPACE2 && deriv == 1) {
    js = left ? A1L_j : A1R_j; ds = left ? A1L_d : A1R_d; cs = left ? A1L_c : A1R_c; nt = 4; den = 4.0;
  } else if (scheme == ORC_AT_SPACE2) {
    js = left ? A2L_j : A2R_j; ds = left ? A2L_d : A2R_d; cs = left ? A2L_c : A2R_c; nt = 6; den = 3.0;
  } else if (deriv == 2) {
    js = left ? S2L_j : S2R_j; ds = left ? S2L_d : S2R_d; cs = left ? S2L_c : S2R_c; nt = 4; den = 2.0;
  } else {
    return 0;
  }
  for (int t = 0; t < nt; ++t) {
    out[t].j = js[t];
    out[t].l = ds[t] ? k : 0;
    out[t].c = cs[t] / (den * dxd);
  }
  return nt;
}

/* Taps of one derivative (deriv = 1 or 2) at a point at position pos (0..S-1) of its PE along
 * one axis.  use_pe = 0 means the axis has no PE boundary.  kL / kR are the effective delays of the
 * PE's left / right buffer points.  Returns the number of taps written to out (at most 32). */
int orc_taps(int order, int scheme, int deriv, int64_t pos, int64_t S, int use_pe, int kL, int kR,
             double dx, orc_tap *out) {
  const int h = order / 2;
  const double *num;
  double den;
  cd_table(order, deriv, &num, &den);
  const double scale = den * dxpow(dx, deriv);
  const int left = use_pe && pos < h;
  const int right = use_pe && pos >= S - h;
  const int k = left ? kL : (right ? kR : 0);
  int nt = 0;
  if ((left || right) && k > 0 && (scheme == ORC_AT_SPACE2 || scheme == ORC_AT_SPACE1))
    return space_expanded_taps(scheme, deriv, left, k, dxpow(dx, deriv), out);
  if ((!left && !right) || scheme == ORC_SYNC || k == 0) {
    /* synchronous: Eq. "general_deriv" */
    for (int j = -h; j <= h; ++j) {
      if (num[j + h] == 0.0) continue;
      out[nt].j = j; out[nt].l = 0; out[nt].c = num[j + h] / scale; ++nt;
    }
    return nt;
  }
  if (scheme == ORC_ASYNC_STD) {
    /* Eq. "general_deriv_async": buffer points at level n-k */
    for (int j = -h; j <= h; ++j) {
      if (num[j + h] == 0.0) continue;
      int buf = (pos + j < 0) || (pos + j >= S);
      out[nt].j = j; out[nt].l = buf ? k : 0; out[nt].c = num[j + h] / scale; ++nt;
    }
    return nt;
  }
  if (order == 2) {
    const double kk = (double)k;
    if (left && deriv == 1) {
      /* (1,2,2)b left: (U_{i+1} - (k+1) U_{i-1}^{n-k} + k U_{i-1}^{n-k-1}) / (2 dx) */
      out[0].j = 1;  out[0].l = 0;     out[0].c = 1.0 / scale;
      out[1].j = -1; out[1].l = k;     out[1].c = -(kk + 1.0) / scale;
      out[2].j = -1; out[2].l = k + 1; out[2].c = kk / scale;
      return 3;
    }
    if (left && deriv == 2) {
      /* (2,2,2)b left: (U_{i+1} - 2 U_i + (k+1) U_{i-1}^{n-k} - k U_{i-1}^{n-k-1}) / dx^2 */
      out[0].j = 1;  out[0].l = 0;     out[0].c = 1.0 / scale;
      out[1].j = 0;  out[1].l = 0;     out[1].c = -2.0 / scale;
      out[2].j = -1; out[2].l = k;     out[2].c = (kk + 1.0) / scale;
      out[3].j = -1; out[3].l = k + 1; out[3].c = -kk / scale;
      return 4;
    }
    if (right && deriv == 1) {
      /* (1,2,2)b right: ((k+1) U_{i+1}^{n-k} - k U_{i+1}^{n-k-1} - U_{i-1}) / (2 dx) */
      out[0].j = 1;  out[0].l = k;     out[0].c = (kk + 1.0) / scale;
      out[1].j = 1;  out[1].l = k + 1; out[1].c = -kk / scale;
      out[2].j = -1; out[2].l = 0;     out[2].c = -1.0 / scale;
      return 3;
    }
    /* (2,2,2)b right: ((k+1) U_{i+1}^{n-k} - k U_{i+1}^{n-k-1} - 2 U_i + U_{i-1}) / dx^2 */
    out[0].j = 1;  out[0].l = k;     out[0].c = (kk + 1.0) / scale;
    out[1].j = 1;  out[1].l = k + 1; out[1].c = -kk / scale;
    out[2].j = 0;  out[2].l = 0;     out[2].c = -2.0 / scale;
    out[3].j = -1; out[3].l = 0;     out[3].c = 1.0 / scale;
    return 4;
  }
  /* (1,4,2) / (2,4,2) and (2,6,2): sum over m of w_m(k) times the central stencil whose buffer points are
   * read at level n-k-m; points inside the PE stay at level n. */
  double w[4];
  int T = 3;
  if (order == 4) w_order4(k, w);
  else { w_order6(k, w); T = 4; }
  for (int m = 0; m < T; ++m) {
    for (int j = -h; j <= h; ++j) {
      if (num[j + h] == 0.0) continue;
      int buf = (pos + j < 0) || (pos + j >= S);
      out[nt].j = j; out[nt].l = buf ? k + m : 0; out[nt].c = w[m] * num[j + h] / scale; ++nt;
    }
  }
  return nt;
}

/* ------------------------------------------------------------------------ the grid */
static int64_t ntot(const orc_cfg *g) { return g->n[0] * g->n[1] * g->n[2]; }
static int64_t ptot(const orc_cfg *g) { return (int64_t)g->pe[0] * g->pe[1] * g->pe[2]; }
int64_t orc_num_sides(const orc_cfg *g) { return 2 * (int64_t)g->dim * ptot(g); }

int orc_check(const orc_cfg *g) {
  if (g->dim != 1 && g->dim != 3) return -1;
  if (g->order != 2 && g->order != 4 && g->order != 6) return -1;
  if (g->tsteps < 0 || g->tsteps > 3) return -1;
  if (g->scheme < 0 || g->scheme > 4) return -1;
  if (g->scheme >= ORC_AT_SPACE2 && (g->order != 2 || g->tsteps > 1)) return -1; /* Cases 2 and 3: CD2, Euler */
  if (g->burgers != 0 && (g->burgers != 1 || g->dim != 1 || g->c[0] != 0.0 || g->scheme > ORC_AT)) return -1;
  if (g->scheme == ORC_AT_SPACE1 && (g->c[0] != 0.0 || g->c[1] != 0.0 || g->c[2] != 0.0)) return -1;
  if (g->L < 1 || g->L > 8) return -1;
  if (g->nmodes < 1) return -1;
  for (int a = 0; a < 3; ++a) {
    if (a >= g->dim && (g->n[a] != 1 || g->pe[a] != 1)) return -1;
    if (g->n[a] < 1 || g->pe[a] < 1 || g->n[a] % g->pe[a] != 0) return -1;
    if (a < g->dim && g->n[a] / g->pe[a] < g->order) return -1; /* S >= 2h */
  }
  return 0;
}

/* the periodic domain has length 2 pi (Sec. 5.1) */
static const double ORC_TWO_PI = 6.283185307179586476925286766559005768;
static double grid_dx(const orc_cfg *g, int a) { return ORC_TWO_PI / (double)g->n[a]; }

/* Eq. "IC": u(x,0) = sum_kappa A sin(kappa x + phi), a product of such sums over the axes in 3D */
void orc_initial(const orc_cfg *g, double *u) {
  const int64_t nx = g->n[0], ny = g->n[1], nz = g->n[2];
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        int64_t idx[3] = {x, y, z};
        double v = 1.0;
        for (int a = 0; a < g->dim; ++a) {
          double xa = (double)idx[a] * grid_dx(g, a);
          double s = 0.0;
          for (int q = 0; q < g->nmodes; ++q) {
            int o = a * g->nmodes + q;
            s = s + g->amp[o] * sin((double)g->kappa[o] * xa + g->phase[o]);
          }
          v = v * s;
        }
        u[(z * ny + y) * nx + x] = v;
      }
}

/* Eq. "ana_sol", with the travelling phase read as kappa (x - c t):
 * u_a = prod_axes sum_kappa A exp(-alpha kappa^2 t) sin(kappa (x - c t) + phi) */
void orc_analytic(const orc_cfg *g, double t, double *u) {
  const int64_t nx = g->n[0], ny = g->n[1], nz = g->n[2];
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        int64_t idx[3] = {x, y, z};
        double v = 1.0;
        for (int a = 0; a < g->dim; ++a) {
          double xa = (double)idx[a] * grid_dx(g, a);
          double s = 0.0;
          for (int q = 0; q < g->nmodes; ++q) {
            int o = a * g->nmodes + q;
            double kap = (double)g->kappa[o];
            s = s + g->amp[o] * exp(-g->alpha * kap * kap * t) * sin(kap * (xa - g->c[a] * t) + g->phase[o]);
          }
          v = v * s;
        }
        u[(z * ny + y) * nx + x] = v;
      }
}

/* the taps of derivative `deriv` along axis a at grid point (x,y,z), given the effective delays */
static int point_taps(const orc_cfg *g, const int32_t *keff, int64_t x, int64_t y, int64_t z, int a, int deriv,
                      orc_tap *taps) {
  int64_t idx[3] = {x, y, z};
  int64_t S[3], p[3];
  for (int b = 0; b < 3; ++b) { S[b] = g->n[b] / g->pe[b]; p[b] = idx[b] / S[b]; }
  int64_t pe_id = (p[2] * g->pe[1] + p[1]) * g->pe[0] + p[0];
  int64_t side0 = 2 * (int64_t)g->dim * pe_id + 2 * a;
  int kL = keff[side0], kR = keff[side0 + 1];
  return orc_taps(g->order, g->scheme, deriv, idx[a] % S[a], S[a], g->pe[a] > 1, kL, kR, grid_dx(g, a), taps);
}

static int64_t wrap_add(int64_t i, int64_t j, int64_t n) {
  int64_t r = (i + j) % n;
  return r < 0 ? r + n : r;
}

static double eval_taps(const orc_cfg *g, const double *const *lev, int64_t x, int64_t y, int64_t z, int a,
                        const orc_tap *taps, int nt) {
  const int64_t nx = g->n[0], ny = g->n[1];
  double s = 0.0;
  for (int t = 0; t < nt; ++t) {
    int64_t q[3] = {x, y, z};
    q[a] = wrap_add(q[a], taps[t].j, g->n[a]);
    s = s + taps[t].c * lev[taps[t].l][(q[2] * ny + q[1]) * nx + q[0]];
  }
  return s;
}

/* Right-hand side f^n = sum_axes ( -c_a D1_a U + alpha D2_a U ) at point pt, with the AT stencils at PE edges;
 * lev[m] = U^{n-m} (m = 0.. as deep as the delays need), keff = effective delay of every PE side. */
static double rhs_point(const orc_cfg *g, const double *const *lev, const int32_t *keff, int64_t pt) {
  const int64_t nx = g->n[0], ny = g->n[1];
  const int64_t x = pt % nx, y = (pt / nx) % ny, z = pt / (nx * ny);
  orc_tap taps[32];
  double f = 0.0;
  for (int a = 0; a < g->dim; ++a) {
    int nt1 = point_taps(g, keff, x, y, z, a, 1, taps);
    double d1 = eval_taps(g, lev, x, y, z, a, taps, nt1);
    int nt2 = point_taps(g, keff, x, y, z, a, 2, taps);
    double d2 = eval_taps(g, lev, x, y, z, a, taps, nt2);
    const double beta1 = g->burgers ? lev[0][pt] : g->c[a];  /* Burgers: the advecting speed is u itself */
    f = f + (-beta1 * d1 + g->alpha * d2);
  }
  return f;
}

/* The right-hand side at every point. */
int orc_rhs(const orc_cfg *g, const double *const *lev, const int32_t *keff, double *f_out) {
  if (orc_check(g)) return -1;
  const int64_t N = ntot(g);
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads)
#endif
  for (int64_t pt = 0; pt < N; ++pt) f_out[pt] = rhs_point(g, lev, keff, pt);
  return 0;
}

/* One forward-Euler step, Eq. "time_disc" with one level: U^{n+1} = U^n + dt f^n. */
int orc_step(const orc_cfg *g, const double *const *lev, const int32_t *keff, double *out) {
  if (orc_check(g)) return -1;
  const int64_t N = ntot(g);
  double *f = (double *)malloc(sizeof(double) * (size_t)N);
  if (!f) return -2;
  orc_rhs(g, lev, keff, f);
  for (int64_t pt = 0; pt < N; ++pt) out[pt] = lev[0][pt] + g->dt * f[pt];
  free(f);
  return 0;
}

/* Adams-Bashforth weights (Eq. "time_disc"; Eq. "time_ab2" for two levels; the three-level weights are the
 * textbook ones): beta[m] multiplies f^{n-m}.  A run starts with fewer levels: Euler, then AB2, then AB3. */
static int ab_weights(int levels, double beta[3]) {
  if (levels <= 1) { beta[0] = 1.0; return 1; }
  if (levels == 2) { beta[0] = 1.5; beta[1] = -0.5; return 2; }
  beta[0] = 23.0 / 12.0; beta[1] = -16.0 / 12.0; beta[2] = 5.0 / 12.0;
  return 3;
}

/* Draw the delays of step n for every PE side (raw, logged) and clamp them (effective). */
static void draw_delays(const orc_cfg *g, int64_t n, int T, uint8_t *raw_out, int32_t *keff) {
  const int64_t nb = orc_num_sides(g);
  for (int64_t b = 0; b < nb; ++b) {
    int k = g->scheme == ORC_SYNC ? 0 : orc_delay_raw(g->seed, n, b, g->L, g->thresholds);
    if (raw_out) raw_out[b] = (uint8_t)k;
    keff[b] = orc_delay_effective(k, n, T);
  }
}

/* Raw delays of steps 0..nsteps-1 for every PE side (step-major), without running the solver. */
int orc_delay_log(const orc_cfg *g, int64_t nsteps, uint8_t *log) {
  if (orc_check(g) || nsteps < 0) return -1;
  const int64_t nb = orc_num_sides(g);
  const int T = orc_time_width(g->order, g->scheme);
  int32_t *keff = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
  if (!keff) return -2;
  for (int64_t n = 0; n < nsteps; ++n) draw_delays(g, n, T, log + n * nb, keff);
  free(keff);
  return 0;
}

/* Full run: initial condition (Eq. "IC", or u0 when given), then nsteps steps.  u_out receives U^{nsteps}.  delay_log (optional)
 * receives the raw delays, nsteps x num_sides bytes, step-major.  history (optional) receives
 * U^0..U^{nsteps}, (nsteps+1) x Ntot doubles.  Time levels are kept in R = L + T slots, level m in
 * slot m mod R. */
int orc_run(const orc_cfg *g, const double *u0, int64_t nsteps, double *u_out, uint8_t *delay_log, double *history) {
  if (orc_check(g) || nsteps < 0) return -1;
  const int T = orc_time_width(g->order, g->scheme);
  const int R = g->L + T;
  const int ts = g->tsteps < 1 ? 1 : g->tsteps;
  const int64_t N = ntot(g), nb = orc_num_sides(g);
  double *ring = (double *)malloc(sizeof(double) * (size_t)(R * N));
  double *fring = (double *)malloc(sizeof(double) * (size_t)(ts * N));
  int32_t *keff = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
  const double **lev = (const double **)malloc(sizeof(double *) * (size_t)R);
  if (!ring || !fring || !keff || !lev) { free(ring); free(fring); free(keff); free(lev); return -2; }
  if (u0) memcpy(ring, u0, sizeof(double) * (size_t)N); else orc_initial(g, ring);
  if (history) memcpy(history, ring, sizeof(double) * (size_t)N);
  /* Multistep start (paper silent): from Eq. "IC" the right-hand sides of the ts-1 levels before t = 0 are
   * those of the analytic solution at t = -m dt (synchronous stencils), so every step uses the full-order
   * weights; from a caller's field, and for Burgers' equation (no analytic solution), the run starts with Euler,
   * then AB2. */
  int prehistory = 0;
  if (ts > 1 && !u0 && !g->burgers) {
    int32_t *zero = (int32_t *)calloc((size_t)nb, sizeof(int32_t));
    double *ua = (double *)malloc(sizeof(double) * (size_t)N);
    if (!zero || !ua) { free(zero); free(ua); free(ring); free(fring); free(keff); free(lev); return -2; }
    for (int m = 1; m < ts; ++m) {
      orc_analytic(g, -(double)m * g->dt, ua);
      const double *l0[1] = {ua};
      orc_rhs(g, l0, zero, fring + ((ts - m) % ts) * N);
    }
    free(zero); free(ua);
    prehistory = 1;
  }
  for (int64_t n = 0; n < nsteps; ++n) {
    draw_delays(g, n, T, delay_log ? delay_log + n * nb : NULL, keff);
    for (int m = 0; m < R - 1; ++m) lev[m] = (n - m >= 0) ? ring + ((n - m) % R) * N : NULL;
    double *next = ring + ((n + 1) % R) * N;
    if (ts == 1) {
      orc_step(g, lev, keff, next);
    } else {
      /* U^{n+1} = U^n + dt sum_m beta_m f^{n-m} */
      orc_rhs(g, lev, keff, fring + (n % ts) * N);
      double beta[3];
      const int nl = ab_weights(prehistory ? ts : (int)(n + 1 < ts ? n + 1 : ts), beta);
      for (int64_t pt = 0; pt < N; ++pt) {
        double sum = 0.0;
        for (int m = 0; m < nl; ++m) sum = sum + beta[m] * fring[(((n - m) % ts + ts) % ts) * N + pt];
        next[pt] = lev[0][pt] + g->dt * sum;
      }
    }
    if (history) memcpy(history + (n + 1) * N, next, sizeof(double) * (size_t)N);
  }
  memcpy(u_out, ring + (nsteps % R) * N, sizeof(double) * (size_t)N);
  free(ring); free(fring); free(keff); free(lev);
  return 0;
}

/* U^{nsteps} at the cells pos[0..npos-1] of a 1D run from Eq. "IC" (forward Euler or Adams-Bashforth), computed only
 * inside their domain of dependence.  Every stencil of the method (central, AT rows, rows expanded in space) reads
 * cells at most reach = max(h, 3) away at the current or delayed levels (Sec. 2, Tables "atschemes-left/right"),
 * and the Adams-Bashforth sum reads the cell's own earlier right-hand sides, so U^{n+1}_i needs only cells within
 * reach of i, and the cells within reach (nsteps - n - 1) of a sampled cell are the only ones stepped at step n
 * (the analytic pre-history of a multistep run is formed on the whole grid, as orc_run does).  Each stepped value is
 * computed by the same operations as in orc_run, so the samples equal orc_run's field bit for bit, at a cost that
 * grows with nsteps^2 instead of N nsteps.  Returns -1 for 3D runs. */
int orc_run_samples(const orc_cfg *g, int64_t nsteps, int64_t npos, const int64_t *pos, double *u_out) {
  if (orc_check(g) || nsteps < 0 || npos < 0 || g->dim != 1) return -1;
  const int T = orc_time_width(g->order, g->scheme);
  const int R = g->L + T;
  const int ts = g->tsteps < 1 ? 1 : g->tsteps;
  const int64_t N = g->n[0], nb = orc_num_sides(g);
  const int64_t reach = g->order / 2 > 3 ? g->order / 2 : 3;
  for (int64_t q = 0; q < npos; ++q)
    if (pos[q] < 0 || pos[q] >= N) return -1;
  double *ring = (double *)malloc(sizeof(double) * (size_t)(R * N));
  double *fring = (double *)malloc(sizeof(double) * (size_t)(ts * N));
  int32_t *keff = (int32_t *)malloc(sizeof(int32_t) * (size_t)nb);
  const double **lev = (const double **)malloc(sizeof(double *) * (size_t)R);
  if (!ring || !fring || !keff || !lev) { free(ring); free(fring); free(keff); free(lev); return -2; }
  orc_initial(g, ring);
  int prehistory = 0;
  if (ts > 1 && !g->burgers) {  /* the same start as orc_run from Eq. "IC" */
    int32_t *zero = (int32_t *)calloc((size_t)nb, sizeof(int32_t));
    double *ua = (double *)malloc(sizeof(double) * (size_t)N);
    if (!zero || !ua) { free(zero); free(ua); free(ring); free(fring); free(keff); free(lev); return -2; }
    for (int m = 1; m < ts; ++m) {
      orc_analytic(g, -(double)m * g->dt, ua);
      const double *l0[1] = {ua};
      orc_rhs(g, l0, zero, fring + ((ts - m) % ts) * N);
    }
    free(zero); free(ua);
    prehistory = 1;
  }
  for (int64_t n = 0; n < nsteps; ++n) {
    draw_delays(g, n, T, NULL, keff);
    for (int m = 0; m < R - 1; ++m) lev[m] = (n - m >= 0) ? ring + ((n - m) % R) * N : NULL;
    double *next = ring + ((n + 1) % R) * N;
    double beta[3];
    const int nl = ts == 1 ? 1 : ab_weights(prehistory ? ts : (int)(n + 1 < ts ? n + 1 : ts), beta);
    const int64_t w = reach * (nsteps - n - 1);
    for (int64_t q = 0; q < npos; ++q) {
      const int64_t width = 2 * w + 1 < N ? 2 * w + 1 : N;
      for (int64_t c = 0; c < width; ++c) {
        const int64_t i = wrap_add(pos[q], c - (width < N ? w : pos[q]), N);
        if (ts == 1) {
          next[i] = lev[0][i] + g->dt * rhs_point(g, lev, keff, i);
        } else {
          fring[(n % ts) * N + i] = rhs_point(g, lev, keff, i);
          double sum = 0.0;
          for (int m = 0; m < nl; ++m) sum = sum + beta[m] * fring[(((n - m) % ts + ts) % ts) * N + i];
          next[i] = lev[0][i] + g->dt * sum;
        }
      }
    }
  }
  for (int64_t q = 0; q < npos; ++q) u_out[q] = ring[(nsteps % R) * N + pos[q]];
  free(ring); free(fring); free(keff); free(lev);
  return 0;
}

/* Sec. 4 averages of E = U - u_a at step n (t = n dt), Sec. 5.1:
 * out = {rms over I, max |E|, mean |E|, mean E, rms over I_I, rms over I_B, rms of u_a, N_I, N_B}.
 * I_B = points within the stencil half-width of a PE boundary along some split axis. */
int orc_error_stats(const orc_cfg *g, const double *u, int64_t n, double *out) {
  if (orc_check(g)) return -1;
  const int64_t N = ntot(g), nx = g->n[0], ny = g->n[1], nz = g->n[2];
  const int h = g->order / 2;
  double *ua = (double *)malloc(sizeof(double) * (size_t)N);
  if (!ua) return -2;
  orc_analytic(g, (double)n * g->dt, ua);
  double s2 = 0.0, smax = 0.0, sabs = 0.0, s1 = 0.0, s2I = 0.0, s2B = 0.0, sa2 = 0.0;
  int64_t nI = 0, nB = 0;
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        int64_t i = (z * ny + y) * nx + x;
        int64_t idx[3] = {x, y, z};
        int inB = 0;
        for (int a = 0; a < g->dim; ++a) {
          int64_t S = g->n[a] / g->pe[a], pos = idx[a] % S;
          if (g->pe[a] > 1 && (pos < h || pos >= S - h)) inB = 1;
        }
        double e = u[i] - ua[i];
        s2 = s2 + e * e;
        sabs = sabs + fabs(e);
        s1 = s1 + e;
        if (fabs(e) > smax) smax = fabs(e);
        sa2 = sa2 + ua[i] * ua[i];
        if (inB) { s2B = s2B + e * e; nB++; } else { s2I = s2I + e * e; nI++; }
      }
  out[0] = sqrt(s2 / (double)N);
  out[1] = smax;
  out[2] = sabs / (double)N;
  out[3] = s1 / (double)N;
  out[4] = nI ? sqrt(s2I / (double)nI) : 0.0;
  out[5] = nB ? sqrt(s2B / (double)nB) : 0.0;
  out[6] = sqrt(sa2 / (double)N);
  out[7] = (double)nI;
  out[8] = (double)nB;
  free(ua);
  return 0;
}

/* Adjoint of J = 1/2 || U^{nsteps} - u_target ||^2 with respect to U^0 and alpha, with the same delays
 * as the forward run (which starts from u0, or from Eq. "IC" when u0 is NULL).  The forward history is stored in full (small grids only); the backward sweep is
 * the literal transpose of orc_step: every tap c * U^{n-l}_{i+j} of point i at step n sends
 * lambda^{n+1}_i * dt * (-c_a or alpha) * c to lambda^{n-l}_{i+j}, and lambda^{n+1}_i reaches
 * lambda^n_i through the identity part of the Euler step.  dJ/dalpha = sum_n dt <lambda^{n+1}, D2 U>. */
/* The adjoint of an Adams-Bashforth run started from a caller's field (Euler, then AB2, then AB3; a run from
 * Eq. "IC" takes its earliest right-hand sides from the analytic solution, which depends on alpha, and is not
 * covered): U^{n+1} = U^n + dt sum_m beta_m f^{n-m} is transposed literally.  Going back from the last step, step n
 * adds lambda^{n+1} to lambda^n (identity) and dt beta_m lambda^{n+1} to the adjoint of f^{n-m}; the adjoint of f^n is
 * then complete and goes back through the taps of f^n to the levels it reads, and dJ/dalpha gains
 * <adjoint of f^n, sum_a D2_a U>. */
static int orc_adjoint_ab(const orc_cfg *g, const double *u0, int64_t nsteps, const double *u_target,
                          double *grad_u0, double *grad_alpha, double *J) {
  if (!u0 && !g->burgers) return -1; /* Burgers' runs always start with Euler (no analytic pre-history) */
  const int ts = g->tsteps;
  const int T = orc_time_width(g->order, g->scheme);
  const int64_t N = ntot(g), nb = orc_num_sides(g);
  const int64_t nx = g->n[0], ny = g->n[1], nz = g->n[2];
  double *hist = (double *)malloc(sizeof(double) * (size_t)((nsteps + 1) * N));
  double *adj = (double *)calloc((size_t)((nsteps + 1) * N), sizeof(double));
  double *adjf = (double *)calloc((size_t)((nsteps > 0 ? nsteps : 1) * N), sizeof(double));
  int32_t *keff = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nsteps > 0 ? nsteps * nb : 1));
  double *ulast = (double *)malloc(sizeof(double) * (size_t)N);
  if (!hist || !adj || !adjf || !keff || !ulast) {
    free(hist); free(adj); free(adjf); free(keff); free(ulast);
    return -2;
  }
  if (orc_run(g, u0, nsteps, ulast, NULL, hist)) {
    free(hist); free(adj); free(adjf); free(keff); free(ulast);
    return -1;
  }
  for (int64_t n = 0; n < nsteps; ++n) draw_delays(g, n, T, NULL, keff + n * nb);
  double jj = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    double r = hist[nsteps * N + i] - u_target[i];
    jj = jj + 0.5 * r * r;
    adj[nsteps * N + i] = r;
  }
  double ga = 0.0;
  for (int64_t n = nsteps - 1; n >= 0; --n) {
    const int32_t *kn = keff + n * nb;
    double beta[3];
    const int nl = ab_weights((int)(n + 1 < ts ? n + 1 : ts), beta);
    for (int64_t i = 0; i < N; ++i) {
      const double lam = adj[(n + 1) * N + i];
      adj[n * N + i] = adj[n * N + i] + lam;
      for (int m = 0; m < nl; ++m) adjf[(n - m) * N + i] = adjf[(n - m) * N + i] + g->dt * beta[m] * lam;
    }
    for (int64_t z = 0; z < nz; ++z)
      for (int64_t y = 0; y < ny; ++y)
        for (int64_t x = 0; x < nx; ++x) {
          int64_t i = (z * ny + y) * nx + x;
          const double af = adjf[n * N + i];
          for (int a = 0; a < g->dim; ++a) {
            orc_tap taps[32];
            for (int deriv = 1; deriv <= 2; ++deriv) {
              int nt = point_taps(g, kn, x, y, z, a, deriv, taps);
              double fac = deriv == 1 ? (g->burgers ? -hist[n * N + i] : -g->c[a]) : g->alpha;
              double dd = 0.0;
              for (int t = 0; t < nt; ++t) {
                int64_t q[3] = {x, y, z};
                q[a] = wrap_add(q[a], taps[t].j, g->n[a]);
                int64_t src = (q[2] * ny + q[1]) * nx + q[0];
                int64_t level = n - taps[t].l;
                adj[level * N + src] = adj[level * N + src] + af * fac * taps[t].c;
                dd = dd + taps[t].c * hist[level * N + src];
              }
              if (deriv == 2) ga = ga + af * dd;
              if (deriv == 1 && g->burgers) adj[n * N + i] = adj[n * N + i] - af * dd;
            }
          }
        }
  }
  memcpy(grad_u0, adj, sizeof(double) * (size_t)N);
  *grad_alpha = ga;
  *J = jj;
  free(hist); free(adj); free(adjf); free(keff); free(ulast);
  return 0;
}

int orc_adjoint(const orc_cfg *g, const double *u0, int64_t nsteps, const double *u_target, double *grad_u0,
                double *grad_alpha, double *J) {
  if (orc_check(g) || nsteps < 0) return -1;
  if (g->tsteps > 1) return orc_adjoint_ab(g, u0, nsteps, u_target, grad_u0, grad_alpha, J);
  const int T = orc_time_width(g->order, g->scheme);
  const int64_t N = ntot(g), nb = orc_num_sides(g);
  const int64_t nx = g->n[0], ny = g->n[1], nz = g->n[2];
  double *hist = (double *)malloc(sizeof(double) * (size_t)((nsteps + 1) * N));
  double *adj = (double *)calloc((size_t)((nsteps + 1) * N), sizeof(double));
  int32_t *keff = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nsteps > 0 ? nsteps * nb : 1));
  double *ulast = (double *)malloc(sizeof(double) * (size_t)N);
  if (!hist || !adj || !keff || !ulast) { free(hist); free(adj); free(keff); free(ulast); return -2; }
  if (orc_run(g, u0, nsteps, ulast, NULL, hist)) { free(hist); free(adj); free(keff); free(ulast); return -1; }
  for (int64_t n = 0; n < nsteps; ++n) draw_delays(g, n, T, NULL, keff + n * nb);
  double jj = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    double r = hist[nsteps * N + i] - u_target[i];
    jj = jj + 0.5 * r * r;
    adj[nsteps * N + i] = r;
  }
  double ga = 0.0;
  for (int64_t n = nsteps - 1; n >= 0; --n) {
    const int32_t *kn = keff + n * nb;
    double *lam_next = adj + (n + 1) * N;
    for (int64_t z = 0; z < nz; ++z)
      for (int64_t y = 0; y < ny; ++y)
        for (int64_t x = 0; x < nx; ++x) {
          int64_t i = (z * ny + y) * nx + x;
          double lam = lam_next[i];
          adj[n * N + i] = adj[n * N + i] + lam;
          for (int a = 0; a < g->dim; ++a) {
            orc_tap taps[32];
            for (int deriv = 1; deriv <= 2; ++deriv) {
              int nt = point_taps(g, kn, x, y, z, a, deriv, taps);
              /* Burgers: f = -U_i^n D1 U + alpha D2 U; the D1 taps carry -U_i^n, and U_i^n itself gets -D1 U */
              double fac = deriv == 1 ? (g->burgers ? -hist[n * N + i] : -g->c[a]) : g->alpha;
              double dd = 0.0;
              for (int t = 0; t < nt; ++t) {
                int64_t q[3] = {x, y, z};
                q[a] = wrap_add(q[a], taps[t].j, g->n[a]);
                int64_t src = (q[2] * ny + q[1]) * nx + q[0];
                int64_t level = n - taps[t].l;
                adj[level * N + src] = adj[level * N + src] + lam * g->dt * fac * taps[t].c;
                dd = dd + taps[t].c * hist[level * N + src];
              }
              if (deriv == 2) ga = ga + lam * g->dt * dd;
              if (deriv == 1 && g->burgers) adj[n * N + i] = adj[n * N + i] - lam * g->dt * dd;
            }
          }
        }
  }
  memcpy(grad_u0, adj, sizeof(double) * (size_t)N);
  *grad_alpha = ga;
  *J = jj;
  free(hist); free(adj); free(keff); free(ulast);
  return 0;
}
