// coeffs.cpp -- derivation of asynchrony-tolerant (AT) finite-difference coefficients in exact
// rational arithmetic (arXiv:1702.00496, Sec. 3).  Host-only code of the C ABI.
//
//  at_coeffs         two-stage derivation of Sec. 3.3 / Example 3: symmetric-pair central weights,
//                    then per-delay time-level weights; expanded result re-checked against Eq. "cond".
//  at_stencil_taps   expanded taps c~_{j,l} (Eq. "general_deriv_at2") built from at_coeffs.
//  at_solve_stencil  single-system derivation of Sec. 3.1-3.2 with the rank tests of Sec. 3.2
//                    (used for Examples 1 and 2 and any user stencil).
//  the stencils expanded in space ((1,2,2)a, (2,2,2)a, (2,1,2); Cases 3 and 2) are derived from their shapes by
//  the same single-system procedure, for the edge point of each side.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/at.h"
#include "internal.h"

namespace {

typedef __int128 i128;

bool g_overflow = false;

i128 iabs(i128 v) { return v < 0 ? -v : v; }
i128 igcd(i128 a, i128 b) {
  a = iabs(a); b = iabs(b);
  while (b != 0) { i128 t = a % b; a = b; b = t; }
  return a;
}
i128 mul_chk(i128 a, i128 b) {
  i128 r;
  if (__builtin_mul_overflow(a, b, &r)) { g_overflow = true; return 0; }
  return r;
}
i128 add_chk(i128 a, i128 b) {
  i128 r;
  if (__builtin_add_overflow(a, b, &r)) { g_overflow = true; return 0; }
  return r;
}

// A reduced fraction num/den with den > 0.
struct Q {
  i128 n, d;
  Q(i128 a = 0, i128 b = 1) : n(a), d(b) { norm(); }
  void norm() {
    if (d < 0) { n = -n; d = -d; }
    if (d == 0) { g_overflow = true; d = 1; }
    i128 g = igcd(n, d);
    if (g > 1) { n /= g; d /= g; }
  }
  bool zero() const { return n == 0; }
};
Q operator+(const Q &a, const Q &b) {
  i128 g = igcd(a.d, b.d);
  i128 db = b.d / g;
  return Q(add_chk(mul_chk(a.n, db), mul_chk(b.n, a.d / g)), mul_chk(a.d, db));
}
Q operator-(const Q &a) { return Q(-a.n, a.d); }
Q operator-(const Q &a, const Q &b) { return a + (-b); }
Q operator*(const Q &a, const Q &b) {
  i128 g1 = igcd(a.n, b.d), g2 = igcd(b.n, a.d);
  if (g1 == 0) g1 = 1;
  if (g2 == 0) g2 = 1;
  return Q(mul_chk(a.n / g1, b.n / g2), mul_chk(a.d / g2, b.d / g1));
}
Q operator/(const Q &a, const Q &b) { return a * Q(b.d, b.n); }
bool operator==(const Q &a, const Q &b) { return a.n == b.n && a.d == b.d; }
double qd(const Q &a) { return (double)a.n / (double)a.d; }

Q qpow(Q b, int e) {
  Q r(1);
  for (int i = 0; i < e; ++i) r = r * b;
  return r;
}
i128 fact(int p) {
  i128 r = 1;
  for (int i = 2; i <= p; ++i) r *= i;
  return r;
}

// Row reduction of [A | b] (rows x (cols+1)).  Returns rank(A) and rank(A|b); x receives the solution
// when rank(A) == rank(A|b) == cols.
void solve_rank(std::vector<std::vector<Q>> m, int cols, int *rankA, int *rankAb, std::vector<Q> *x) {
  const int rows = (int)m.size();
  int r = 0;
  std::vector<int> pivcol;
  for (int c = 0; c < cols && r < rows; ++c) {
    int p = -1;
    for (int i = r; i < rows; ++i)
      if (!m[i][c].zero()) { p = i; break; }
    if (p < 0) continue;
    std::swap(m[p], m[r]);
    Q inv = Q(1) / m[r][c];
    for (int k = c; k <= cols; ++k) m[r][k] = m[r][k] * inv;
    for (int i = 0; i < rows; ++i) {
      if (i == r || m[i][c].zero()) continue;
      Q f = m[i][c];
      for (int k = c; k <= cols; ++k) m[i][k] = m[i][k] - f * m[r][k];
    }
    pivcol.push_back(c);
    ++r;
  }
  *rankA = r;
  int extra = 0;
  for (int i = r; i < rows; ++i)
    if (!m[i][cols].zero()) extra = 1;
  *rankAb = r + extra;
  if (x) {
    x->assign(cols, Q(0));
    if (extra == 0 && r == cols)
      for (int i = 0; i < r; ++i) (*x)[pivcol[i]] = m[i][cols];
  }
}

int time_width(int d, int a) {
  int T = 1;
  for (int q = 1; 2 * q < d + a; ++q) ++T;
  return T;
}

struct Derived {
  int h, T;
  std::vector<Q> cd;               // 2h+1 per-point central weights
  std::vector<Q> phi;              // h+1 symmetric-pair weights
  std::vector<std::vector<Q>> w;   // [L][T]
};

int derive(int d, int a, int L, Derived *out) {
  const int h = a / 2;
  // Stage 1 (Eq. "general_deriv_cds"): unknowns phi_j on the pair u_{i+j} + (-1)^d u_{i-j}; its Taylor
  // coefficient of u^(p) dx^p / p! is j^p (1 + (-1)^(d+p)), so only rows with p + d even survive.
  const int j0 = (d % 2 == 0) ? 0 : 1;
  std::vector<std::vector<Q>> m;
  for (int p = 0; p < d + a; ++p) {
    if ((p + d) % 2) continue;
    std::vector<Q> row;
    for (int j = j0; j <= h; ++j) {
      Q e = (j == 0) ? Q(p == 0 ? 2 : 0) : Q(2) * qpow(Q(j), p) / Q(fact(p));
      row.push_back(e);
    }
    row.push_back(Q(p == d ? 1 : 0));
    m.push_back(row);
  }
  const int cols = h - j0 + 1;
  int rA, rAb;
  std::vector<Q> phi;
  solve_rank(m, cols, &rA, &rAb, &phi);
  if (rA != rAb) return AT_ERR_INCONSISTENT;
  if (rA < cols) return AT_ERR_SINGULAR;
  out->h = h;
  out->phi.assign(h + 1, Q(0));
  for (int j = j0; j <= h; ++j) out->phi[j] = phi[j - j0];
  out->cd.assign(2 * h + 1, Q(0));
  const Q sgn = (d % 2 == 0) ? Q(1) : Q(-1);
  for (int j = 1; j <= h; ++j) {
    out->cd[h + j] = out->phi[j];
    out->cd[h - j] = sgn * out->phi[j];
  }
  out->cd[h] = (d % 2 == 0) ? Q(2) * out->phi[0] : Q(0);
  // Stage 2 (Example 3): the copies of the stage-1 stencil read at levels n-k-m, m < T, are combined with
  // weights that cancel the asynchronous rows q = 1..T-1 (their p-dependence factors out, Eq. "cond-async2"):
  //   sum_m w_m (k+m)^q = delta_{q0}.
  const int T = time_width(d, a);
  out->T = T;
  out->w.assign(L, std::vector<Q>(T, Q(0)));
  for (int k = 0; k < L; ++k) {
    std::vector<std::vector<Q>> v;
    for (int q = 0; q < T; ++q) {
      std::vector<Q> row;
      for (int mm = 0; mm < T; ++mm) row.push_back(qpow(Q(k + mm), q));
      row.push_back(Q(q == 0 ? 1 : 0));
      v.push_back(row);
    }
    std::vector<Q> wk;
    solve_rank(v, T, &rA, &rAb, &wk);
    if (rA != rAb) return AT_ERR_INCONSISTENT;
    if (rA < T) return AT_ERR_SINGULAR;
    out->w[k] = wk;
  }
  return g_overflow ? AT_ERR_ARG : AT_OK;
}

struct Tap {
  int j, l;
  Q c;
};

// Eq. "cond" with dt ~ dx^2 on an explicit stencil {(j_t, l_t)}: the single system of Sec. 3.1-3.2, rows
// p + 2q < d + a.  Returns AT_OK with the unique coefficients, or the rank-test status.
int solve_shape(int d, int a, const std::vector<int> &js, const std::vector<int> &ls, std::vector<Q> *x) {
  std::vector<std::vector<Q>> m;
  for (int p = 0; p < d + a; ++p)
    for (int q = 0; p + 2 * q < d + a; ++q) {
      std::vector<Q> row;
      for (size_t t = 0; t < js.size(); ++t) row.push_back(qpow(Q(js[t]), p) * qpow(Q(-ls[t]), q) / Q(fact(p) * fact(q)));
      row.push_back(Q((p == d && q == 0) ? 1 : 0));
      m.push_back(row);
    }
  int rA, rAb;
  solve_rank(m, (int)js.size(), &rA, &rAb, x);
  if (rA != rAb) return AT_ERR_INCONSISTENT;
  if (rA < (int)js.size()) return AT_ERR_SINGULAR;
  return g_overflow ? AT_ERR_ARG : AT_OK;
}

// Shapes of the rows expanded in space at the edge point whose buffer points lie on the left (side 0): points
// with flag 1 are buffer points, read at level n-k.  The right edge (side 1) uses the mirror image.
//   (1,2,2)a: {i+1, i; i-1, i-2}      (2,2,2)a: {i+2, i+1, i; i-1, i-2, i-3}      (2,1,2): {i+1, i; i-1, i-2}
// Returns the order a of the row, or 0 if the scheme defines no row for this derivative.
int space_shape(int scheme, int d, std::vector<int> *js, std::vector<int> *buf) {
  if (scheme == AT_AT_SPACE2 && d == 1) { *js = {1, 0, -1, -2}; *buf = {0, 0, 1, 1}; return 2; }
  if (scheme == AT_AT_SPACE2 && d == 2) { *js = {2, 1, 0, -1, -2, -3}; *buf = {0, 0, 0, 1, 1, 1}; return 2; }
  if (scheme == AT_AT_SPACE1 && d == 2) { *js = {1, 0, -1, -2}; *buf = {0, 0, 1, 1}; return 1; }
  return 0;
}

// The row expanded in space of derivative d at the edge point of `side` for delay k >= 1, derived from its
// shape.  Returns AT_OK, AT_ERR_ARG (no row for this derivative) or the rank-test status.
int space_taps(int scheme, int d, int k, int side, std::vector<Tap> *taps) {
  std::vector<int> js, buf;
  const int a = space_shape(scheme, d, &js, &buf);
  if (a == 0) return AT_ERR_ARG;
  std::vector<int> ls(js.size());
  for (size_t t = 0; t < js.size(); ++t) {
    if (side == 1) js[t] = -js[t];
    ls[t] = buf[t] ? k : 0;
  }
  std::vector<Q> x;
  const int rc = solve_shape(d, a, js, ls, &x);
  if (rc != AT_OK) return rc;
  taps->clear();
  for (size_t t = 0; t < js.size(); ++t)
    if (!x[t].zero()) taps->push_back(Tap{js[t], ls[t], x[t]});
  return AT_OK;
}

// Taps of the stencil at a point `pos` cells in from the edge whose buffer points lie on `side`.
void expand(const Derived &D, int scheme, int k, int pos, int side, std::vector<Tap> *taps) {
  const int h = D.h;
  taps->clear();
  auto add = [&](int j, int l, Q c) {
    if (c.zero()) return;
    for (auto &t : *taps)
      if (t.j == j && t.l == l) { t.c = t.c + c; return; }
    taps->push_back(Tap{j, l, c});
  };
  auto is_buf = [&](int j) { return side == 0 ? (pos + j < 0) : (j > pos); };
  if (scheme == AT_SYNC || k == 0) {
    for (int j = -h; j <= h; ++j) add(j, 0, D.cd[h + j]);
  } else if (scheme == AT_ASYNC_STD) {
    for (int j = -h; j <= h; ++j) add(j, is_buf(j) ? k : 0, D.cd[h + j]);
  } else {
    for (int mm = 0; mm < D.T; ++mm)
      for (int j = -h; j <= h; ++j) add(j, is_buf(j) ? k + mm : 0, D.w[k][mm] * D.cd[h + j]);
  }
  std::vector<Tap> kept;
  for (auto &t : *taps)
    if (!t.c.zero()) kept.push_back(t);
  *taps = kept;
}

// Eq. "cond" with dt ~ dx^2: sum c~ j^p (-l)^q / (p! q!) = [ (p,q) == (d,0) ] for p + 2q < d + a.
bool check_cond(const std::vector<Tap> &taps, int d, int a) {
  for (int p = 0; p <= d + a; ++p)
    for (int q = 0; p + 2 * q < d + a; ++q) {
      Q s(0);
      for (auto &t : taps) s = s + t.c * qpow(Q(t.j), p) * qpow(Q(-t.l), q);
      s = s / Q(fact(p) * fact(q));
      Q want((p == d && q == 0) ? 1 : 0);
      if (!(s == want)) return false;
    }
  return true;
}

thread_local char g_err[256] = "";

}  // namespace

void at_internal_set_error(const char *msg) {
  std::snprintf(g_err, sizeof(g_err), "%s", msg);
}

extern "C" const char *at_last_error(void) { return g_err; }

extern "C" int at_coeffs(int32_t deriv, int32_t order, int32_t L, at_coeffs_t *out) {
  if (!out || (deriv != 1 && deriv != 2) || (order != 2 && order != 4 && order != 6) || L < 1 || L > 8) {
    at_internal_set_error("at_coeffs: deriv must be 1|2, order 2|4|6, 1 <= L <= 8, out non-NULL");
    return AT_ERR_ARG;
  }
  g_overflow = false;
  Derived D;
  int rc = derive(deriv, order, L, &D);
  if (rc != AT_OK) {
    at_internal_set_error("at_coeffs: derivation failed (rank test or overflow)");
    return rc;
  }
  // Re-check the expanded scheme at every edge position and delay against Eq. "cond".
  std::vector<Tap> taps;
  for (int k = 0; k < L; ++k)
    for (int side = 0; side < 2; ++side)
      for (int pos = 0; pos < D.h; ++pos) {
        expand(D, AT_AT, k, pos, side, &taps);
        if (!check_cond(taps, deriv, order)) {
          at_internal_set_error("at_coeffs: expanded scheme violates the Taylor conditions");
          return AT_ERR_INCONSISTENT;
        }
      }
  if (g_overflow) {
    at_internal_set_error("at_coeffs: rational overflow");
    return AT_ERR_ARG;
  }
  std::memset(out, 0, sizeof(*out));
  out->deriv = deriv; out->order = order; out->L = L; out->h = D.h; out->T = D.T;
  i128 den = 1;
  for (auto &q : D.cd) den = den / igcd(den, q.d) * q.d;
  out->cd_den = (int64_t)den;
  for (int j = 0; j <= 2 * D.h; ++j) {
    out->cd[j] = qd(D.cd[j]);
    out->cd_num[j] = (int64_t)(D.cd[j].n * (den / D.cd[j].d));
  }
  for (int j = 0; j <= D.h; ++j) out->phi[j] = qd(D.phi[j]);
  for (int k = 0; k < L; ++k) {
    i128 wd = 1;
    for (auto &q : D.w[k]) wd = wd / igcd(wd, q.d) * q.d;
    out->w_den[k] = (int64_t)wd;
    for (int mm = 0; mm < D.T; ++mm) {
      out->w[k][mm] = qd(D.w[k][mm]);
      out->w_num[k][mm] = (int64_t)(D.w[k][mm].n * (wd / D.w[k][mm].d));
    }
  }
  return AT_OK;
}

extern "C" int at_stencil_taps(int32_t deriv, int32_t order, int32_t scheme, int32_t k, int32_t pos, int32_t side,
                               int32_t cap, int32_t *j_out, int32_t *l_out, double *c_out, int32_t *ntaps) {
  if ((deriv != 1 && deriv != 2) || (order != 2 && order != 4 && order != 6) || scheme < 0 || scheme > 4 || k < 0 || k > 7 ||
      pos < 0 || side < 0 || side > 1 || cap < 0 || !j_out || !l_out || !c_out || !ntaps) {
    at_internal_set_error("at_stencil_taps: bad argument");
    return AT_ERR_ARG;
  }
  const bool space = scheme == AT_AT_SPACE2 || scheme == AT_AT_SPACE1;
  if (space && order != 2) {
    at_internal_set_error("at_stencil_taps: the rows expanded in space are second-order schemes (order 2)");
    return AT_ERR_ARG;
  }
  g_overflow = false;
  Derived D;
  int rc = derive(deriv, order, k + 1, &D);
  if (rc != AT_OK) return rc;
  std::vector<Tap> taps;
  if (space && k > 0 && pos == 0) {
    if ((rc = space_taps(scheme, deriv, k, side, &taps)) != AT_OK) {
      at_internal_set_error("at_stencil_taps: (2,1,2) defines no first derivative, or the row's system failed");
      return rc;
    }
  } else {
    expand(D, space ? AT_SYNC : scheme, k, pos, side, &taps);
  }
  if ((int)taps.size() > cap) {
    at_internal_set_error("at_stencil_taps: cap too small");
    return AT_ERR_ARG;
  }
  for (size_t t = 0; t < taps.size(); ++t) {
    j_out[t] = taps[t].j; l_out[t] = taps[t].l; c_out[t] = qd(taps[t].c);
  }
  *ntaps = (int32_t)taps.size();
  return AT_OK;
}

extern "C" int at_solve_stencil(int32_t deriv, int32_t order, int32_t r, int32_t npts, const int32_t *j,
                                const int32_t *l, int64_t *num_out, int64_t *den_out, double *c_out,
                                int32_t *rank_out) {
  if (deriv < 1 || deriv > 4 || order < 1 || order > 8 || r < 1 || r > 4 || npts < 1 || npts > 32 || !j || !l ||
      !num_out || !den_out || !c_out || !rank_out) {
    at_internal_set_error("at_solve_stencil: bad argument");
    return AT_ERR_ARG;
  }
  g_overflow = false;
  std::vector<std::vector<Q>> m;
  const int lim = deriv + order;
  for (int p = 0; p < lim; ++p)
    for (int q = 0; p + r * q < lim; ++q) {
      std::vector<Q> row;
      for (int i = 0; i < npts; ++i) row.push_back(qpow(Q(j[i]), p) * qpow(Q(-l[i]), q) / Q(fact(p) * fact(q)));
      row.push_back(Q((p == deriv && q == 0) ? 1 : 0));
      m.push_back(row);
    }
  int rA, rAb;
  std::vector<Q> x;
  solve_rank(m, npts, &rA, &rAb, &x);
  *rank_out = rA;
  if (g_overflow) {
    at_internal_set_error("at_solve_stencil: rational overflow");
    return AT_ERR_ARG;
  }
  if (rA != rAb) {
    at_internal_set_error("at_solve_stencil: rank(A) != rank(A|b): the stencil gives no scheme");
    return AT_ERR_INCONSISTENT;
  }
  if (rA < npts) {
    at_internal_set_error("at_solve_stencil: rank deficient: infinitely many schemes");
    return AT_ERR_SINGULAR;
  }
  for (int i = 0; i < npts; ++i) {
    num_out[i] = (int64_t)x[i].n;
    den_out[i] = (int64_t)x[i].d;
    c_out[i] = qd(x[i]);
  }
  return AT_OK;
}
