// api.cu -- the solver handle of the C ABI (include/at.h): configuration checks, merged stencil
// coefficients, ring-buffer bookkeeping, step driver and error statistics.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/at.h"
#include "internal.h"
#include "philox.cuh"



namespace {

const double kTwoPi = 6.283185307179586476925286766559005768;

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

int time_width(const at_config_t *c) { return c->scheme == AT_AT ? c->order / 2 + 1 : 1; }

// Time levels of the integrator: 1 (forward Euler), 2 (AB2) or 3 (AB3); 0 means 1.
int time_levels(const at_config_t *c) { return c->tsteps < 2 ? 1 : c->tsteps; }

int check_config(const at_config_t *c) {
  if (!c) return fail(AT_ERR_ARG, "config is NULL");
  if (c->dim != 1 && c->dim != 3) return fail(AT_ERR_ARG, "dim must be 1 or 3");
  if (c->order != 2 && c->order != 4 && c->order != 6) return fail(AT_ERR_ARG, "order must be 2, 4 or 6");
  if (c->tsteps < 0 || c->tsteps > 3) return fail(AT_ERR_ARG, "tsteps must be 0..3");
  if (c->scheme < AT_SYNC || c->scheme > AT_AT_SPACE1)
    return fail(AT_ERR_ARG, "scheme must be AT_SYNC, AT_ASYNC_STD, AT_AT, AT_AT_SPACE2 or AT_AT_SPACE1");
  if (c->scheme >= AT_AT_SPACE2 && (c->order != 2 || c->tsteps > 1))
    return fail(AT_ERR_ARG, "the rows expanded in space are second-order schemes with forward Euler (Cases 2, 3)");
  if (c->burgers != 0 && (c->burgers != 1 || c->dim != 1 || c->c[0] != 0.0 || c->scheme > AT_AT))
    return fail(AT_ERR_ARG, "burgers: 1D, c = 0 (the advecting speed is u) and scheme AT_SYNC, AT_ASYNC_STD or AT_AT");
  if (c->scheme == AT_AT_SPACE1 && (c->c[0] != 0.0 || c->c[1] != 0.0 || c->c[2] != 0.0))
    return fail(AT_ERR_ARG, "(2,1,2) gives only a second derivative: AT_AT_SPACE1 needs c = 0 (diffusion)");
  if (c->L < 1 || c->L > AT_MAX_L) return fail(AT_ERR_ARG, "L must be in 1..8");
  if (c->nmodes < 1 || c->nmodes > AT_MAX_MODES) return fail(AT_ERR_ARG, "nmodes must be in 1..16");
  if (!c->amp || !c->phase || !c->kappa) return fail(AT_ERR_ARG, "amp, phase and kappa are required");
  int64_t tot = 1;
  for (int a = 0; a < 3; ++a) {
    if (c->n[a] < 1 || c->pe[a] < 1) return fail(AT_ERR_ARG, "n and pe must be positive");
    if (a >= c->dim && (c->n[a] != 1 || c->pe[a] != 1)) return fail(AT_ERR_ARG, "unused axes must have n = pe = 1");
    if (c->n[a] % c->pe[a]) return fail(AT_ERR_ARG, "n must be a multiple of pe on every axis");
    if (a < c->dim && c->n[a] / c->pe[a] < c->order) return fail(AT_ERR_ARG, "PE width must be at least the order (2h)");
    if (c->n[a] > (int64_t)1 << 30) return fail(AT_ERR_ARG, "n too large");
    tot *= c->n[a];
  }
  if (tot > ((int64_t)1 << 31) - 1) return fail(AT_ERR_ARG, "more than 2^31-1 points");
  if (!(c->dt > 0.0) || !std::isfinite(c->dt) || !std::isfinite(c->alpha)) return fail(AT_ERR_ARG, "dt must be positive and finite");
  if (c->thresholds) {
    for (int m = 0; m + 1 < c->L; ++m) {
      if (c->thresholds[m] > ((uint64_t)1 << 32)) return fail(AT_ERR_ARG, "thresholds must lie in [0, 2^32]");
      if (m > 0 && c->thresholds[m] < c->thresholds[m - 1]) return fail(AT_ERR_ARG, "thresholds must ascend");
    }
  }
  return AT_OK;
}

int64_t sides_of(const at_config_t *c) { return 2 * (int64_t)c->dim * c->pe[0] * c->pe[1] * c->pe[2]; }

}  // namespace

extern "C" int at_ring_slots(const at_config_t *cfg, int32_t *R) {
  int rc = check_config(cfg);
  if (rc) return rc;
  if (!R) return fail(AT_ERR_ARG, "R is NULL");
  const int ts = time_levels(cfg);
  *R = cfg->L + time_width(cfg) + (ts > 1 ? ts - 1 : 0);
  return AT_OK;
}

extern "C" int at_num_sides(const at_config_t *cfg, int64_t *sides) {
  int rc = check_config(cfg);
  if (rc) return rc;
  if (!sides) return fail(AT_ERR_ARG, "sides is NULL");
  *sides = sides_of(cfg);
  return AT_OK;
}

extern "C" int at_delay(uint64_t seed, int64_t step, int64_t side, int32_t L, const uint64_t *thresholds_host) {
  if (L < 1 || L > AT_MAX_L || step < 0 || side < 0) return fail(AT_ERR_ARG, "at_delay: bad argument");
  return atfd::delay_draw(seed, (uint32_t)step, (uint32_t)side, L, thresholds_host);
}

// The merged edge rows of axis a for the schemes expanded in space: D1 and D2 rows from at_stencil_taps (derived
// from their shapes), checked to be the same for every delay 1..L-1, merged as dt (-c_a D1/dx + alpha D2/dx^2).
static int space_rows(const at_config_t *cfg, int a, double dx, StepParams *p) {
  for (int side = 0; side < 2; ++side) {
    int n = 0;
    for (int deriv = 1; deriv <= 2; ++deriv) {
      if (deriv == 1 && cfg->scheme == AT_AT_SPACE1) continue;  // diffusion only
      int32_t j0[16], l0[16], nt0 = 0;
      double c0[16];
      for (int k = 1; k < cfg->L; ++k) {
        int32_t jj[16], ll[16], nt = 0;
        double cc[16];
        int rc = at_stencil_taps(deriv, cfg->order, cfg->scheme, k, 0, side, 16, jj, ll, cc, &nt);
        if (rc != AT_OK) return rc;
        if (k == 1) {
          nt0 = nt;
          for (int t = 0; t < nt; ++t) { j0[t] = jj[t]; l0[t] = ll[t] ? 1 : 0; c0[t] = cc[t]; }
        } else {
          bool same = nt == nt0;
          for (int t = 0; same && t < nt; ++t) same = jj[t] == j0[t] && (ll[t] ? 1 : 0) == l0[t] && cc[t] == c0[t];
          if (!same) return fail(AT_ERR_INCONSISTENT, "edge row coefficients depend on the delay");
        }
      }
      const double scale = deriv == 1 ? -cfg->c[a] / dx : cfg->alpha / (dx * dx);
      for (int t = 0; t < nt0; ++t) {
        int slot = -1;
        for (int u = 0; u < n; ++u)
          if (p->ej[a][side][u] == j0[t] && p->ebuf[a][side][u] == l0[t]) slot = u;
        if (slot < 0) {
          if (n == AT_MAX_ETAPS) return fail(AT_ERR_ARG, "edge row has too many taps");
          slot = n++;
          p->ej[a][side][slot] = (int8_t)j0[t];
          p->ebuf[a][side][slot] = (int8_t)l0[t];
          p->ec[a][side][slot] = 0.0;
          p->eq[a][side][slot] = 0.0;
        }
        p->ec[a][side][slot] += cfg->dt * scale * c0[t];
        if (deriv == 2) p->eq[a][side][slot] += cfg->dt * c0[t] / (dx * dx);
      }
    }
    p->ecount[a][side] = n;
  }
  return AT_OK;
}

int at_prepare_params(const at_config_t *cfg, double *ring_dev, uint8_t *log_dev, int64_t log_steps, StepParams *out) {
  int rc = check_config(cfg);
  if (rc) return rc;
  const int T = time_width(cfg);
  const int h = cfg->order / 2;
  at_coeffs_t c1, c2;
  if ((rc = at_coeffs(1, cfg->order, cfg->L, &c1)) != AT_OK) return rc;
  if ((rc = at_coeffs(2, cfg->order, cfg->L, &c2)) != AT_OK) return rc;
  if (cfg->scheme == AT_AT && (c1.T != T || c2.T != T)) return fail(AT_ERR_INCONSISTENT, "time widths of D1 and D2 differ");
  StepParams &p = *out;
  std::memset(&p, 0, sizeof(p));
  p.ring = ring_dev;
  p.log = log_dev;
  p.log_steps = log_dev ? log_steps : 0;
  p.ntot = cfg->n[0] * cfg->n[1] * cfg->n[2];
  p.nb = sides_of(cfg);
  p.dim = cfg->dim; p.h = h; p.T = T; p.R = cfg->L + T; p.L = cfg->L; p.scheme = cfg->scheme;
  p.ts = time_levels(cfg);
  p.burgers = cfg->burgers;
  p.frhs = p.ts > 1 && ring_dev ? ring_dev + (int64_t)p.R * p.ntot : nullptr;
  // Adams-Bashforth weights of dt f^{n-m} with l = 1, 2, 3 stored levels (Eq. "time_ab2" for two levels; the
  // three-level weights are the standard ones)
  const double beta[3][3] = {{1.0, 0.0, 0.0}, {1.5, -0.5, 0.0}, {23.0 / 12.0, -16.0 / 12.0, 5.0 / 12.0}};
  std::memcpy(p.beta, beta, sizeof(beta));
  p.seed = cfg->seed;
  p.use_thr = cfg->thresholds != nullptr;
  if (cfg->thresholds)
    for (int m = 0; m + 1 < cfg->L; ++m) p.thr[m] = cfg->thresholds[m];
  double s0 = p.ts > 1 ? 0.0 : 1.0, q0 = 0.0;
  for (int a = 0; a < 3; ++a) {
    p.n[a] = (int32_t)cfg->n[a];
    p.pe[a] = cfg->pe[a];
    p.S[a] = (int32_t)(cfg->n[a] / cfg->pe[a]);
    p.use_pe[a] = (a < cfg->dim && cfg->pe[a] > 1) ? 1 : 0;
    if (a >= cfg->dim) continue;
    const double dx = kTwoPi / (double)cfg->n[a];
    for (int j = -h; j <= h; ++j) {
      const double v = cfg->dt * (-cfg->c[a] * c1.cd[j + h] / dx + cfg->alpha * c2.cd[j + h] / (dx * dx));
      const double dv = cfg->dt * c2.cd[j + h] / (dx * dx);
      if (j == 0) { s0 += v; q0 += dv; p.sc[a] = v; p.qc[a] = dv; } else { p.s[a][j + h] = v; p.q[a][j + h] = dv; }
      if (a == 0) {
        p.b1[j + h] = cfg->dt * c1.cd[j + h] / dx;
        p.b2[j + h] = cfg->dt * cfg->alpha * c2.cd[j + h] / (dx * dx);
      }
    }
    if (cfg->scheme >= AT_AT_SPACE2 && cfg->pe[a] > 1 && (rc = space_rows(cfg, a, dx, &p)) != AT_OK) return rc;
  }
  p.s0 = s0;
  p.q0 = q0;
  for (int k = 0; k < cfg->L; ++k)
    for (int m = 0; m < T; ++m)
      p.w[k][m] = cfg->scheme == AT_AT ? c2.w[k][m] : (m == 0 ? 1.0 : 0.0);
  return AT_OK;
}

// Start of an Adams-Bashforth history.  With the analytic initial condition the right-hand sides of the ts-1
// levels before t = 0 are those of the analytic solution at t = -m dt with central differences (the paper does
// not say how its multistep runs start; this keeps every step at the full order); from a caller's field the run
// starts with forward Euler and raises the order as right-hand sides accumulate.  Ring slot 1 (level 1, which
// the first step writes) holds the analytic field meanwhile.
static cudaError_t ab_start(at_handle *hd, bool analytic) {
  const StepParams &p = hd->sp;
  if (p.ts <= 1) return cudaSuccess;
  const int ns = p.ts - 1;
  hd->sp.ab_steady = analytic ? 0 : ns;
  cudaError_t e = cudaSuccess;
  if (analytic) {
    double *tmp = p.ring + p.ntot;
    for (int m = 1; m < p.ts && e == cudaSuccess; ++m) {
      const int slot = ((-m) % ns + ns) % ns;
      e = launch_wave_field(hd->wp, -(double)m * hd->cfg.dt, hd->d_tables, tmp, hd->stream);
      if (e == cudaSuccess) e = launch_sync_rhs(p, tmp, p.frhs + (int64_t)slot * p.ntot, hd->stream);
    }
  }
  if (e == cudaSuccess) e = launch_step_counter(hd->d_step + 1, analytic ? -(int64_t)ns : 0, true, hd->stream);
  return e;
}

extern "C" int at_init(const at_config_t *cfg, double *ring_dev, int64_t ring_len, uint8_t *log_dev,
                       int64_t log_steps, void *stream, at_handle_t **out) {
  int rc = check_config(cfg);
  if (rc) return rc;
  if (!out || !ring_dev) return fail(AT_ERR_ARG, "ring_dev and out are required");
  if (log_steps < 0 || (log_steps > 0 && !log_dev)) return fail(AT_ERR_ARG, "log_dev required when log_steps > 0");
  int32_t R = 0;
  at_ring_slots(cfg, &R);
  const int64_t ntot = cfg->n[0] * cfg->n[1] * cfg->n[2];
  if (ring_len < (int64_t)R * ntot) return fail(AT_ERR_ARG, "ring_len < R * points (R from at_ring_slots)");

  at_handle *hd = new (std::nothrow) at_handle();
  if (!hd) return fail(AT_ERR_ARG, "out of host memory");
  if ((rc = at_prepare_params(cfg, ring_dev, log_steps > 0 ? log_dev : nullptr, log_steps, &hd->sp)) != AT_OK) {
    delete hd;
    return rc;
  }
  hd->cfg = *cfg;
  if (cfg->thresholds) hd->thr.assign(cfg->thresholds, cfg->thresholds + (cfg->L - 1));
  hd->cfg.thresholds = nullptr;
  hd->cfg.amp = hd->cfg.phase = nullptr;
  hd->cfg.kappa = nullptr;
  hd->stream = (cudaStream_t)stream;
  hd->log_steps = log_steps;
  StepParams &p = hd->sp;

  WaveParams &w = hd->wp;
  std::memset(&w, 0, sizeof(w));
  w.dim = cfg->dim; w.nmodes = cfg->nmodes; w.alpha = cfg->alpha;
  for (int a = 0; a < 3; ++a) {
    w.n[a] = (int32_t)cfg->n[a];
    w.dx[a] = kTwoPi / (double)cfg->n[a];
    w.xpi[a] = 2.0 / (double)cfg->n[a];
    w.c[a] = cfg->c[a];
    if (a >= cfg->dim) continue;
    for (int q = 0; q < cfg->nmodes; ++q) {
      w.amp[a][q] = cfg->amp[a * cfg->nmodes + q];
      w.phase[a][q] = cfg->phase[a * cfg->nmodes + q];
      w.kappa[a][q] = (double)cfg->kappa[a * cfg->nmodes + q];
    }
  }

  const size_t n_tables = (size_t)(cfg->n[0] + cfg->n[1] + cfg->n[2]);
  const size_t keff_bytes = (size_t)(2 * p.nb + 255) / 256 * 256;
  // 3D grouped shapes: visit interior groups first, then edge groups, so a warp's lanes share one path
  std::vector<int32_t> order;
  int64_t n_interior = 0;
  if (cfg->dim == 3 && cfg->n[0] % 4 == 0 && (p.use_pe[0] == 0 || p.S[0] % 4 == 0)) {
    const int64_t gx = cfg->n[0] / 4, groups = ntot / 4;
    const int h = cfg->order / 2;
    auto interior = [&](int64_t g) {  // every cell and stencil neighbour inside the group's PE and the domain
      const int64_t r = g / gx;
      const int x0 = (int)(g - r * gx) * 4, z = (int)(r / cfg->n[1]), y = (int)(r - (int64_t)z * cfg->n[1]);
      const int c[3] = {x0, y, z}, span[3] = {3, 0, 0};
      for (int a = 0; a < 3; ++a) {
        if (c[a] - h < 0 || c[a] + span[a] + h >= cfg->n[a]) return false;
        const int pos = c[a] % p.S[a];
        if (p.use_pe[a] && (pos < h || pos + span[a] >= p.S[a] - h)) return false;
      }
      return true;
    };
    // edge groups sorted by how they meet the PE faces (counting sort, g ascending within a kind): the x faces
    // the group touches, and per y and z axis the cell count into the lower / upper face region, so a warp's
    // lanes mostly take the same branches
    const int nc = 2 * h + 1;
    auto axis_kind = [&](int a, int c) {
      if (!p.use_pe[a]) return 0;
      const int pos = c % p.S[a];
      if (pos < h) return h - pos;
      if (pos > p.S[a] - 1 - h) return h + pos - (p.S[a] - 1 - h);
      return 0;
    };
    auto kind = [&](int64_t g) {
      const int64_t r = g / gx;
      const int x0 = (int)(g - r * gx) * 4, z = (int)(r / cfg->n[1]), y = (int)(r - (int64_t)z * cfg->n[1]);
      int xt = 0;
      if (p.use_pe[0]) xt = (x0 % p.S[0] == 0 ? 1 : 0) | (x0 % p.S[0] + 4 == p.S[0] ? 2 : 0);
      return (xt * nc + axis_kind(1, y)) * nc + axis_kind(2, z);
    };
    order.reserve((size_t)groups);
    std::vector<int64_t> start((size_t)(4 * nc * nc + 1), 0);
    for (int64_t g = 0; g < groups; ++g) {
      if (interior(g)) order.push_back((int32_t)g);
      else ++start[(size_t)kind(g) + 1];
    }
    n_interior = (int64_t)order.size();
    for (size_t k = 1; k < start.size(); ++k) start[k] += start[k - 1];
    order.resize((size_t)groups);
    for (int64_t g = 0; g < groups; ++g)
      if (!interior(g)) order[(size_t)(n_interior + start[(size_t)kind(g)]++)] = (int32_t)g;
  }
  const size_t order_bytes = (order.size() * sizeof(int32_t) + 255) / 256 * 256;
  const size_t bytes = 512 + keff_bytes + order_bytes +
                       sizeof(double) * ((size_t)AT_STAT_BLOCKS * AT_STAT_FIELDS + 16 + n_tables);
  cudaError_t e = cudaMalloc(&hd->scratch, bytes);
  if (e != cudaSuccess) { delete hd; return cuda_fail(e, "at_init: cudaMalloc"); }
  char *base = (char *)hd->scratch;
  hd->d_step = (int64_t *)(base + 256);
  p.keff = (uint8_t *)(base + 512);
  p.order = order.empty() ? nullptr : (const int32_t *)(base + 512 + keff_bytes);
  hd->n_interior = n_interior;
  hd->d_partials = (double *)(base + 512 + keff_bytes + order_bytes);
  if (!order.empty() &&
      (e = cudaMemcpy((void *)p.order, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice)) !=
          cudaSuccess) {
    cudaFree(hd->scratch);
    delete hd;
    return cuda_fail(e, "at_init: group order");
  }
  hd->d_result = hd->d_partials + (size_t)AT_STAT_BLOCKS * AT_STAT_FIELDS;
  hd->d_tables = hd->d_result + 16;
  p.status = nullptr;
  p.ab_first = hd->d_step + 1;
  fuse_setup(&p, fuse_max_k(p, ring_dev, AT_MAX_FUSE));
  if ((e = launch_wave_field(w, 0.0, hd->d_tables, ring_dev, hd->stream)) != cudaSuccess ||
      (e = ab_start(hd, cfg->burgers == 0)) != cudaSuccess ||
      (e = launch_draw_delays(p, 0, hd->stream)) != cudaSuccess) {
    cudaFree(hd->scratch);
    delete hd;
    return cuda_fail(e, "at_init: initial condition");
  }
  hd->ab_analytic = p.ts > 1 && cfg->burgers == 0;
  *out = hd;
  return AT_OK;
}

// Steps per captured graph: kGraphSteps, rounded down to whole blocks of K steps when at_step runs blocks.
static int64_t graph_steps(const at_handle *hd) {
  const int64_t K = hd->sp.fuse_k;
  return K > 1 ? kGraphSteps / K * K : kGraphSteps;
}

static int build_graph(at_handle *hd) {
  cudaStream_t cap;
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "at_step: capture stream");
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  int64_t g = 0;
  const int64_t K = hd->sp.fuse_k, G = graph_steps(hd);
  for (; K > 1 && g + K <= G && e == cudaSuccess; g += K) e = launch_forward_block(hd->sp, g, hd->d_step, cap);
  for (; g < G && e == cudaSuccess; ++g) e = launch_forward_step(hd->sp, g, hd->d_step, cap);
  if (e == cudaSuccess) e = launch_step_counter(hd->d_step, G, false, cap);
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&hd->exec, graph, 0);
  cudaStreamDestroy(cap);
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    hd->exec = nullptr;
    return cuda_fail(e, "at_step: graph");
  }
  hd->graph = graph;
  return AT_OK;
}

extern "C" int at_step(at_handle_t *hd, int64_t nsteps) {
  if (!hd || nsteps < 0) return fail(AT_ERR_ARG, "at_step: bad argument");
  hd->adj_nsteps = -1;  // stepping on invalidates a recorded adjoint forward pass
  if (hd->sp.log && hd->step + nsteps > hd->log_steps) return fail(AT_ERR_STATE, "at_step: delay log is full");
  if (hd->step + nsteps > 0xFFFFFFFFll) return fail(AT_ERR_STATE, "at_step: step counter exceeds 32 bits");
  cudaError_t e;
  int64_t s = 0;
  // the start of a multistep run from a caller's field, where the weights change from step to step, runs in single
  // launches; the captured graphs hold steps of the steady form
  for (; s < nsteps && hd->sp.ts > 1 && hd->step < hd->sp.ab_steady; ++s) {
    if ((e = launch_forward_step(hd->sp, hd->step, nullptr, hd->stream)) != cudaSuccess)
      return cuda_fail(e, "at_step: launch");
    hd->step += 1;
  }
  const int64_t G = graph_steps(hd), chunks = (nsteps - s) / G;
  if (chunks > 0) {
    if (!hd->exec) {
      int rc = build_graph(hd);
      if (rc) return rc;
    }
    if ((e = launch_step_counter(hd->d_step, hd->step, true, hd->stream)) != cudaSuccess)
      return cuda_fail(e, "at_step: counter");
    for (int64_t c = 0; c < chunks; ++c) {
      if ((e = cudaGraphLaunch(hd->exec, hd->stream)) != cudaSuccess) return cuda_fail(e, "at_step: graph launch");
      hd->step += G;
    }
  }
  s += chunks * G;
  const int64_t K = hd->sp.fuse_k;
  for (; K > 1 && s + K <= nsteps; s += K) {
    if ((e = launch_forward_block(hd->sp, hd->step, nullptr, hd->stream)) != cudaSuccess)
      return cuda_fail(e, "at_step: launch");
    hd->step += K;
  }
  for (; s < nsteps; ++s) {
    if ((e = launch_forward_step(hd->sp, hd->step, nullptr, hd->stream)) != cudaSuccess)
      return cuda_fail(e, "at_step: launch");
    hd->step += 1;
  }
  return AT_OK;
}

extern "C" int at_set_fusion(at_handle_t *hd, int32_t k, int32_t *k_used) {
  if (!hd || k < 1 || k > AT_MAX_FUSE) return fail(AT_ERR_ARG, "at_set_fusion: k must be 1..4");
  cudaError_t e = cudaStreamSynchronize(hd->stream);
  if (e != cudaSuccess) return cuda_fail(e, "at_set_fusion");
  if (hd->exec) cudaGraphExecDestroy(hd->exec);
  if (hd->graph) cudaGraphDestroy(hd->graph);
  hd->exec = nullptr;
  hd->graph = nullptr;
  const int K = fuse_max_k(hd->sp, hd->sp.ring, k);
  fuse_setup(&hd->sp, K);
  if (k_used) *k_used = K;
  return AT_OK;
}

extern "C" int at_reset(at_handle_t *hd, const double *u0_dev) {
  if (!hd) return fail(AT_ERR_ARG, "at_reset: NULL handle");
  cudaError_t e;
  if (u0_dev)
    e = cudaMemcpyAsync(hd->sp.ring, u0_dev, sizeof(double) * (size_t)hd->sp.ntot, cudaMemcpyDeviceToDevice,
                        hd->stream);
  else
    e = launch_wave_field(hd->wp, 0.0, hd->d_tables, hd->sp.ring, hd->stream);
  hd->ab_analytic = hd->sp.ts > 1 && u0_dev == nullptr && hd->cfg.burgers == 0;
  if (e == cudaSuccess) e = ab_start(hd, hd->ab_analytic);
  if (e == cudaSuccess) e = launch_draw_delays(hd->sp, 0, hd->stream);
  if (e != cudaSuccess) return cuda_fail(e, "at_reset");
  hd->step = 0;
  hd->adj_nsteps = -1;  // a recorded adjoint forward pass no longer matches the handle
  return AT_OK;
}

extern "C" int at_set_launch(at_handle_t *hd, int32_t threads, int32_t blocks_per_sm) {
  if (!hd || (threads != 128 && threads != 256 && threads != 512) || blocks_per_sm < 1 || blocks_per_sm > 64)
    return fail(AT_ERR_ARG, "at_set_launch: threads must be 128, 256 or 512 and blocks_per_sm in 1..64");
  cudaError_t e = cudaStreamSynchronize(hd->stream);
  if (e != cudaSuccess) return cuda_fail(e, "at_set_launch");
  if (hd->exec) cudaGraphExecDestroy(hd->exec);
  if (hd->graph) cudaGraphDestroy(hd->graph);
  hd->exec = nullptr;
  hd->graph = nullptr;
  hd->sp.threads = threads;
  hd->sp.blocks_per_sm = blocks_per_sm;
  return AT_OK;
}

extern "C" int at_sync(at_handle_t *hd) {
  if (!hd) return fail(AT_ERR_ARG, "at_sync: NULL handle");
  cudaError_t e = cudaStreamSynchronize(hd->stream);
  if (e != cudaSuccess) return cuda_fail(e, "at_sync");
  return AT_OK;
}

extern "C" int at_state(at_handle_t *hd, int64_t *step, double **field_dev) {
  if (!hd) return fail(AT_ERR_ARG, "at_state: NULL handle");
  if (step) *step = hd->step;
  if (field_dev) *field_dev = hd->sp.ring + (hd->step % hd->sp.R) * hd->sp.ntot;
  return AT_OK;
}

static int finish_stats(at_handle *hd, at_stats_t *out, const char *where);

extern "C" int at_error_stats(at_handle_t *hd, at_stats_t *out) {
  if (!hd || !out) return fail(AT_ERR_ARG, "at_error_stats: bad argument");
  if (hd->cfg.burgers) return fail(AT_ERR_ARG, "at_error_stats: Burgers' equation has no analytic solution here "
                                              "(use at_error_stats_ref with a finer run)");
  const double *u = hd->sp.ring + (hd->step % hd->sp.R) * hd->sp.ntot;
  const double t = (double)hd->step * hd->cfg.dt;
  cudaError_t e = launch_error_stats(hd->wp, hd->sp, u, t, hd->d_tables, hd->d_partials, hd->d_result, hd->stream);
  if (e != cudaSuccess) return cuda_fail(e, "at_error_stats: launch");
  return finish_stats(hd, out, "at_error_stats");
}

extern "C" int at_error_stats_ref(at_handle_t *hd, const double *ref_dev, int32_t refine, at_stats_t *out) {
  if (!hd || !out || !ref_dev || refine < 1) return fail(AT_ERR_ARG, "at_error_stats_ref: bad argument");
  const double *u = hd->sp.ring + (hd->step % hd->sp.R) * hd->sp.ntot;
  cudaError_t e = launch_error_stats_ref(hd->wp, hd->sp, u, ref_dev, refine, hd->d_partials, hd->d_result,
                                         hd->stream);
  if (e != cudaSuccess) return cuda_fail(e, "at_error_stats_ref: launch");
  return finish_stats(hd, out, "at_error_stats_ref");
}

static int finish_stats(at_handle *hd, at_stats_t *out, const char *where) {
  cudaError_t e;
  double r[AT_STAT_FIELDS];
  if ((e = cudaMemcpyAsync(r, hd->d_result, sizeof(r), cudaMemcpyDeviceToHost, hd->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(hd->stream)) != cudaSuccess)
    return cuda_fail(e, where);
  const double N = (double)hd->sp.ntot;
  out->rms = std::sqrt(r[0] / N);
  out->max_abs = r[1];
  out->mean_abs = r[2] / N;
  out->mean = r[3] / N;
  out->rms_I = r[7] > 0 ? std::sqrt(r[4] / r[7]) : 0.0;
  out->rms_B = r[8] > 0 ? std::sqrt(r[5] / r[8]) : 0.0;
  out->ua_rms = std::sqrt(r[6] / N);
  out->n_I = (int64_t)r[7];
  out->n_B = (int64_t)r[8];
  out->step = hd->step;
  if (!std::isfinite(out->rms) || !std::isfinite(out->max_abs)) {
    char buf[120];
    std::snprintf(buf, sizeof(buf), "%s: non-finite error", where);
    return fail(AT_ERR_NONFINITE, buf);
  }
  return AT_OK;
}

extern "C" int at_destroy(at_handle_t *hd) {
  if (!hd) return AT_OK;
  cudaError_t e = cudaStreamSynchronize(hd->stream);
  if (hd->exec) cudaGraphExecDestroy(hd->exec);
  if (hd->graph) cudaGraphDestroy(hd->graph);
  cudaFree(hd->scratch);
  delete hd;
  if (e != cudaSuccess) return cuda_fail(e, "at_destroy");
  return AT_OK;
}
