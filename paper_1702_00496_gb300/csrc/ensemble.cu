// ensemble.cu -- many independent delay realizations of the 1D problem in one persistent launch.
//
// The accuracy claims of the paper are statistical: Sec. 4 defines the error through an ensemble average
// over delay realizations (the overline of Eq. "aveE_split"), and Sec. 5.1 averages runs with different
// initial phases.  This engine runs `count` 1D realizations (each with its own grid size, PE count, delay
// range L, seed and initial condition) to completion inside ONE persistent kernel:
//   - a fixed grid of CTAs pulls realizations from an atomic work counter in longest-first order (the host
//     sorts by cost N * steps), so uneven grid sizes balance across the 152 SMs;
//   - a CTA owns its realization for the whole run: it writes U^0 (Eq. "IC"), advances every step with the
//     same fused stencil as the per-step kernel (delay draw, halo extrapolation, merged taps), separated by
//     __syncthreads, and finally reduces E = U - u_a (Eq. "ana_sol") into the realization's statistics;
//   - a second small kernel forms, per grid size, the ensemble mean and unbiased variance of the RMS error.
// Both kernels and the counter reset are captured once in a CUDA graph; one run is one graph launch.
// Each realization keeps its own R-slot ring in global memory (level m in slot m mod R); small rings stay
// in L1/L2.  Reads use plain coherent loads because the kernel reads back levels it wrote itself.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/at.h"
#include "modes.cuh"
#include "stencil.cuh"

namespace {

struct MemberParams {
  StepParams p;
  double amp[AT_MAX_MODES];        // A of Eq. "IC"
  double amp_final[AT_MAX_MODES];  // A exp(-alpha kappa^2 t_final)
  double amp_pre[2][AT_MAX_MODES]; // Adams-Bashforth pre-history: A exp(alpha kappa^2 m dt), m = 1, 2
  double shift_pre[2];             // and its phase shift c t = -c m dt
  double phase[AT_MAX_MODES];
  double kappa[AT_MAX_MODES];
  double dx, xpi, shift_final;     // grid spacing, 2 / n (point i at x = pi i xpi), c * t_final
  int64_t steps;                   // steps this member runs
  int32_t nmodes, group;           // group: index of the member's summary group
  int32_t twin;                    // member whose final field this one is compared with, or -1
  // the same modes prepared for the recurrences over k (when ms_ic.rot), exactly as the single-problem path
  // prepares them, so a member's fields and statistics carry the same bits: t = 0, t_final, t = -dt, -2 dt
  ModeSet ms_ic, ms_fin, ms_pre[2];
};

constexpr int kStatFields = AT_STAT_FIELDS;

__device__ double wave_1d(const MemberParams &m, const ModeSet &ms, const double *amp, double shift, int i) {
  if (ms.rot) return atfd::mode_sum(ms, m.nmodes, (double)i * m.xpi);
  const double x = (double)i * m.dx;
  double s = 0.0;
  for (int q = 0; q < m.nmodes; ++q) s += amp[q] * sin(m.kappa[q] * (x - shift) + m.phase[q]);
  return s;
}

// Adams-Bashforth pre-history of a realization (the same start as a single problem): dt f of the analytic
// solution at t = -m dt, m = 1..ts-1, with central differences, into the right-hand-side slot of level -m.
// The member's PE split is switched off in the shared parameters meanwhile; ring slot 1 holds the field.
template <int H>
__device__ void member_prehistory(MemberParams &m) {
  const int N = m.p.n[0], ns = m.p.ts - 1;
  double *tmp = m.p.ring + m.p.ntot;
  const int use_pe = m.p.use_pe[0];
  __syncthreads();
  if (threadIdx.x == 0) m.p.use_pe[0] = 0;
  for (int mm = 1; mm <= ns; ++mm) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) tmp[i] = wave_1d(m, m.ms_pre[mm - 1], m.amp_pre[mm - 1], m.shift_pre[mm - 1], i);
    __syncthreads();
    double *out = m.p.frhs + (int64_t)(((-mm) % ns + ns) % ns) * m.p.ntot;
    for (int k = threadIdx.x; k < (N >> 2); k += blockDim.x) {
      double f[4], uc[4];
      atfd::group_eval<1, H, atfd::LdCoherent, false>(m.p, nullptr, tmp, 0, k << 2, 0, 0, f, uc);
      for (int q = 0; q < 4; ++q) out[(k << 2) + q] = f[q];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) m.p.use_pe[0] = use_pe;
  __syncthreads();
}

// One realization, all steps: the delays of step n+1 are drawn (into the other half of the shared delay
// buffer) while step n is computed; one barrier per step publishes both the new level and the new delays.
template <int H, bool AB, bool SPACE>
__device__ void run_member(const StepParams &p, uint8_t *keff_sh, int64_t nsteps) {
  const int groups = p.n[0] >> 2;
  atfd::draw_sides(p, 0, threadIdx.x, blockDim.x, keff_sh);
  __syncthreads();
  for (int64_t n = 0; n < nsteps; ++n) {
    const double *un = p.ring + (n % p.R) * p.ntot;
    double *out = p.ring + ((n + 1) % p.R) * p.ntot;
    if (n + 1 < nsteps) atfd::draw_sides(p, n + 1, threadIdx.x, blockDim.x, keff_sh + ((n + 1) & 1) * p.nb);
    const uint8_t *keff = keff_sh + (n & 1) * p.nb;
    for (int k = threadIdx.x; k < groups; k += blockDim.x)
      if (SPACE && p.scheme >= AT_AT_SPACE2)
        atfd::group_step<1, H, atfd::LdCoherent, AB, 2>(p, keff, un, out, n, (int)(atfd::group_1d_order(p, k) << 2),
                                                        0, 0);
      else
        atfd::group_update<1, H, atfd::LdCoherent, AB>(p, keff, un, out, n, (int)(atfd::group_1d_order(p, k) << 2),
                                                       0, 0);
    __syncthreads();
  }
}

// HMAX: the largest stencil half-width among the members; AB: some member uses Adams-Bashforth; SPACE: some member
// uses rows expanded in space.  The host picks the smallest variant that covers every member, so the common case
// keeps the register budget of the H <= 2 Euler step.
template <int HMAX, bool AB, bool SPACE>
__global__ void __launch_bounds__(1024, 1) ensemble_kernel(const MemberParams *__restrict__ members,
                                                       const int32_t *__restrict__ order, int32_t count,
                                                       int32_t *counter, double *__restrict__ member_stats) {
  __shared__ MemberParams m;
  __shared__ int32_t item;
  __shared__ double red[kStatFields][32];  // one partial per warp
  extern __shared__ uint8_t keff_sh[];  // two buffers of the largest member's side count
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(counter, 1);
    __syncthreads();
    if (item >= count) break;
    const int32_t r = order[item];
    {
      const int words = (int)(sizeof(MemberParams) / sizeof(int32_t));
      const int32_t *src = reinterpret_cast<const int32_t *>(members + r);
      int32_t *dst = reinterpret_cast<int32_t *>(&m);
      for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
    }
    __syncthreads();
    const int N = m.p.n[0];
    for (int i = threadIdx.x; i < N; i += blockDim.x) m.p.ring[i] = wave_1d(m, m.ms_ic, m.amp, 0.0, i);
    __syncthreads();
    if (AB && m.p.ts > 1) {
      if (m.p.h == 1) member_prehistory<1>(m);
      else if (HMAX == 2 || m.p.h == 2) member_prehistory<2>(m);
      else member_prehistory<HMAX>(m);
      if (m.p.h == 1) run_member<1, AB, SPACE>(m.p, keff_sh, m.steps);
      else if (HMAX == 2 || m.p.h == 2) run_member<2, AB, SPACE>(m.p, keff_sh, m.steps);
      else run_member<HMAX, AB, SPACE>(m.p, keff_sh, m.steps);
    } else {
      if (m.p.h == 1) run_member<1, false, SPACE>(m.p, keff_sh, m.steps);
      else if (HMAX == 2 || m.p.h == 2) run_member<2, false, SPACE>(m.p, keff_sh, m.steps);
      else run_member<HMAX, false, SPACE>(m.p, keff_sh, m.steps);
    }
    // statistics of E = U^steps - u_a(x, steps dt), as in the single-problem reduction
    const double *u = m.p.ring + (m.steps % m.p.R) * m.p.ntot;
    double acc[kStatFields];
#pragma unroll
    for (int f = 0; f < kStatFields; ++f) acc[f] = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const double ua = wave_1d(m, m.ms_fin, m.amp_final, m.shift_final, i);
      const int pos = i % m.p.S[0];
      const bool inB = m.p.use_pe[0] && (pos < m.p.h || pos >= m.p.S[0] - m.p.h);
      const double e = u[i] - ua;
      acc[0] += e * e;
      acc[1] = fmax(acc[1], fabs(e));
      acc[2] += fabs(e);
      acc[3] += e;
      if (inB) { acc[5] += e * e; acc[8] += 1.0; } else { acc[4] += e * e; acc[7] += 1.0; }
      acc[6] += ua * ua;
      if (e != e) acc[1] = e;
    }
    // warp partials by shuffles, then warp 0 combines them in warp order (deterministic)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
    for (int f = 0; f < kStatFields; ++f) {
      double v = acc[f];
      for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_down_sync(0xffffffffu, v, o);
        v = (f == 1) ? ((w != w) ? w : fmax(v, w)) : v + w;
      }
      if (lane == 0) red[f][warp] = v;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int f = 0; f < kStatFields; ++f) {
        double v = lane < nwarps ? red[f][lane] : (f == 1 ? 0.0 : 0.0);
        for (int o = 16; o > 0; o >>= 1) {
          const double w = __shfl_down_sync(0xffffffffu, v, o);
          v = (f == 1) ? ((w != w) ? w : fmax(v, w)) : v + w;
        }
        if (lane == 0) red[f][0] = v;
      }
    }
    __syncthreads();
    if (threadIdx.x < kStatFields) member_stats[(int64_t)r * kStatFields + threadIdx.x] = red[threadIdx.x][0];
    __syncthreads();
  }
}

// The member's final field against its twin's: RMS and mean absolute value over the points of U - U_twin (0
// without a twin), into diff[2r], diff[2r+1]; one block per member, the block's partial sums combined in a fixed
// order (deterministic).
__global__ void __launch_bounds__(256) twin_diff_kernel(const MemberParams *__restrict__ members,
                                                        double *__restrict__ diff) {
  __shared__ double red[2][8];
  const MemberParams &a = members[blockIdx.x];
  if (a.twin < 0) {
    if (threadIdx.x < 2) diff[2 * (int64_t)blockIdx.x + threadIdx.x] = 0.0;
    return;
  }
  const MemberParams &b = members[a.twin];
  const double *ua = a.p.ring + (a.steps % a.p.R) * a.p.ntot;
  const double *ub = b.p.ring + (b.steps % b.p.R) * b.p.ntot;
  double s2 = 0.0, s1 = 0.0;
  for (int64_t i = threadIdx.x; i < a.p.ntot; i += blockDim.x) {
    const double d = ua[i] - ub[i];
    s2 = fma(d, d, s2);
    s1 += fabs(d);
  }
  for (int o = 16; o > 0; o >>= 1) {
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s2;
    red[1][threadIdx.x >> 5] = s1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t2 = 0.0, t1 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t2 += red[0][w];
      t1 += red[1][w];
    }
    diff[2 * (int64_t)blockIdx.x] = sqrt(t2 / (double)a.p.ntot);
    diff[2 * (int64_t)blockIdx.x + 1] = t1 / (double)a.p.ntot;
  }
}

constexpr int kGroupFields = 9;

// Per summary group g, summed in member order: mean and unbiased variance of the members' RMS errors, the mean of
// their mean absolute errors, and -- over the members that have a twin -- mean and unbiased variance of the RMS
// and of the mean absolute value of U - U_twin.  out[g] = {rms mean, rms var, count, diff-RMS mean, diff-RMS var,
// members with a twin, diff-abs mean, diff-abs var, mean-abs-error mean}.
__global__ void summary_kernel(const double *__restrict__ member_stats, const double *__restrict__ member_diff,
                               const MemberParams *__restrict__ members, int32_t count, int32_t ngroups,
                               double *__restrict__ out /* [ngroups][kGroupFields] */) {
  for (int g = threadIdx.x; g < ngroups; g += blockDim.x) {
    double s = 0.0, sa = 0.0, c = 0.0, sd = 0.0, sda = 0.0, cd = 0.0;
    for (int r = 0; r < count; ++r)
      if (members[r].group == g) {
        const double N = (double)members[r].p.ntot;
        s += sqrt(member_stats[(int64_t)r * kStatFields] / N);
        sa += member_stats[(int64_t)r * kStatFields + 2] / N;
        c += 1.0;
        if (members[r].twin >= 0) {
          sd += member_diff[2 * (int64_t)r];
          sda += member_diff[2 * (int64_t)r + 1];
          cd += 1.0;
        }
      }
    const double mean = c > 0 ? s / c : 0.0, dmean = cd > 0 ? sd / cd : 0.0, damean = cd > 0 ? sda / cd : 0.0;
    double v = 0.0, vd = 0.0, vda = 0.0;
    for (int r = 0; r < count; ++r)
      if (members[r].group == g) {
        const double d = sqrt(member_stats[(int64_t)r * kStatFields] / (double)members[r].p.ntot) - mean;
        v += d * d;
        if (members[r].twin >= 0) {
          const double e = member_diff[2 * (int64_t)r] - dmean, f = member_diff[2 * (int64_t)r + 1] - damean;
          vd += e * e;
          vda += f * f;
        }
      }
    double *o = out + kGroupFields * (int64_t)g;
    o[0] = mean;
    o[1] = c > 1 ? v / (c - 1.0) : 0.0;
    o[2] = c;
    o[3] = dmean;
    o[4] = cd > 1 ? vd / (cd - 1.0) : 0.0;
    o[5] = cd;
    o[6] = damean;
    o[7] = cd > 1 ? vda / (cd - 1.0) : 0.0;
    o[8] = c > 0 ? sa / c : 0.0;
  }
}

__global__ void reset_counter(int32_t *c) { *c = 0; }

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

const double kTwoPi = 6.283185307179586476925286766559005768;

}  // namespace

struct at_ensemble {
  int32_t count = 0, ngroups = 0;
  cudaStream_t stream = nullptr;
  void *scratch = nullptr;
  MemberParams *d_members = nullptr;
  int32_t *d_order = nullptr;
  int32_t *d_counter = nullptr;
  double *d_member_stats = nullptr;
  double *d_member_diff = nullptr;
  double *d_summary = nullptr;
  std::vector<int64_t> group_key;
  std::vector<int64_t> member_n, member_steps;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int threads = 256, blocks = 0;
  size_t dyn_smem = 0;
};

// Ring and log sizes (in doubles and bytes) the members need, laid out member after member; validates the runs.
extern "C" int at_ensemble_sizes(const at_config_t *members, const at_member_t *runs, int32_t count,
                                 int64_t *ring_len, int64_t *log_len) {
  if (!members || !runs || count < 1 || !ring_len || !log_len) return fail(AT_ERR_ARG, "at_ensemble_sizes: bad argument");
  int64_t ring = 0, log = 0;
  for (int r = 0; r < count; ++r) {
    int32_t R;
    int64_t nb;
    int rc = at_ring_slots(members + r, &R);
    if (rc) return rc;
    if ((rc = at_num_sides(members + r, &nb))) return rc;
    if (members[r].dim != 1 || members[r].n[0] % 4 || (members[r].pe[0] > 1 && (members[r].n[0] / members[r].pe[0]) % 4))
      return fail(AT_ERR_ARG, "ensemble members must be 1D with N and the PE width multiples of 4");
    if (members[r].burgers) return fail(AT_ERR_ARG, "ensemble: Burgers' members are not supported (no analytic error)");
    const at_member_t &u = runs[r];
    if (u.nsteps < 0 || u.nsteps > 0xFFFFFFFFll) return fail(AT_ERR_ARG, "ensemble: nsteps must be in 0..2^32-1");
    if (u.group < -1) return fail(AT_ERR_ARG, "ensemble: group must be >= -1");
    if (u.twin < -1 || u.twin >= count || u.twin == r || (u.twin >= 0 && members[u.twin].n[0] != members[r].n[0]))
      return fail(AT_ERR_ARG, "ensemble: twin must be -1 or another member with the same n[0]");
    ring += (int64_t)R * members[r].n[0];
    log += u.nsteps * nb;
  }
  *ring_len = ring;
  *log_len = log;
  return AT_OK;
}

extern "C" int at_ensemble_create(const at_config_t *members, const at_member_t *runs, int32_t count,
                                  double *ring_dev, int64_t ring_len, uint8_t *log_dev, int64_t log_len,
                                  int32_t threads, int32_t ctas_per_sm, void *stream, at_ensemble_t **out) {
  int64_t need_ring, need_log;
  int rc = at_ensemble_sizes(members, runs, count, &need_ring, &need_log);
  if (rc) return rc;
  if (!out || !ring_dev || ring_len < need_ring) return fail(AT_ERR_ARG, "at_ensemble_create: ring too small");
  if (reinterpret_cast<uintptr_t>(ring_dev) % 16)
    return fail(AT_ERR_ARG, "at_ensemble_create: ring not 16-byte aligned (the group kernels use 16-byte accesses)");
  if (log_dev && log_len < need_log) return fail(AT_ERR_ARG, "at_ensemble_create: log too small");
  if (threads == 0) threads = 1024;
  if (threads != 128 && threads != 256 && threads != 512 && threads != 1024)
    return fail(AT_ERR_ARG, "threads must be 128, 256, 512 or 1024");

  std::vector<MemberParams> host(count);
  std::map<int64_t, int> groups;
  auto key_of = [&](int r) { return runs[r].group >= 0 ? (int64_t)runs[r].group : members[r].n[0]; };
  for (int r = 0; r < count; ++r) groups[key_of(r)] = 0;
  int gi = 0;
  for (auto &kv : groups) kv.second = gi++;
  at_ensemble *e = new (std::nothrow) at_ensemble();
  if (!e) return fail(AT_ERR_ARG, "out of host memory");
  int64_t ring_off = 0, log_off = 0, max_nb = 1;
  for (int r = 0; r < count; ++r) {
    const at_config_t &c = members[r];
    // merged taps, extrapolation weights and delay parameters exactly as for a single problem
    int32_t R;
    int64_t nb;
    at_ring_slots(&c, &R);
    at_num_sides(&c, &nb);
    MemberParams &m = host[r];
    std::memset(&m, 0, sizeof(m));
    const int64_t nsteps = runs[r].nsteps;
    rc = at_prepare_params(&c, ring_dev + ring_off, log_dev ? log_dev + log_off : nullptr, nsteps, &m.p);
    max_nb = std::max<int64_t>(max_nb, nb);
    if (rc) { delete e; return rc; }
    m.nmodes = c.nmodes;
    m.dx = kTwoPi / (double)c.n[0];
    m.xpi = 2.0 / (double)c.n[0];
    const double tf = (double)nsteps * c.dt;
    m.shift_final = c.c[0] * tf;
    for (int q = 0; q < c.nmodes; ++q) {
      m.amp[q] = c.amp[q];
      m.phase[q] = c.phase[q];
      m.kappa[q] = (double)c.kappa[q];
      m.amp_final[q] = tf == 0.0 ? c.amp[q] : c.amp[q] * std::exp(-c.alpha * m.kappa[q] * m.kappa[q] * tf);
      for (int mm = 1; mm <= 2; ++mm)
        m.amp_pre[mm - 1][q] = c.amp[q] * std::exp(c.alpha * m.kappa[q] * m.kappa[q] * (double)mm * c.dt);
    }
    for (int mm = 1; mm <= 2; ++mm) m.shift_pre[mm - 1] = -c.c[0] * (double)mm * c.dt;
    fill_modes(&m.ms_ic, m.amp, m.phase, m.kappa, c.nmodes, c.alpha, c.c[0], 0.0);
    fill_modes(&m.ms_fin, m.amp, m.phase, m.kappa, c.nmodes, c.alpha, c.c[0], tf);
    for (int mm = 1; mm <= 2; ++mm)
      fill_modes(&m.ms_pre[mm - 1], m.amp, m.phase, m.kappa, c.nmodes, c.alpha, c.c[0], -(double)mm * c.dt);
    m.group = groups[key_of(r)];
    m.steps = nsteps;
    m.twin = runs[r].twin;
    e->member_n.push_back(c.n[0]);
    e->member_steps.push_back(nsteps);
    ring_off += (int64_t)R * c.n[0];
    log_off += nsteps * nb;
  }
  for (auto &kv : groups) e->group_key.push_back(kv.first);
  e->count = count;
  e->ngroups = (int32_t)groups.size();
  e->stream = (cudaStream_t)stream;
  e->threads = threads;
  // longest first (cost ~ N * steps): the largest runs start first
  std::vector<int32_t> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (double)members[a].n[0] * (double)runs[a].nsteps > (double)members[b].n[0] * (double)runs[b].nsteps;
  });

  const size_t b_members = sizeof(MemberParams) * (size_t)count;
  const size_t b_order = sizeof(int32_t) * (size_t)count;
  const size_t b_stats = sizeof(double) * (size_t)count * kStatFields;
  const size_t b_diff = sizeof(double) * 2 * (size_t)count;
  const size_t b_sum = sizeof(double) * kGroupFields * (size_t)e->ngroups;
  const size_t b_first = sizeof(int64_t) * (size_t)count;
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  cudaError_t err =
      cudaMalloc(&e->scratch, up(b_members) + up(b_order) + 256 + up(b_stats) + up(b_diff) + up(b_sum) + up(b_first));
  if (err != cudaSuccess) { delete e; return cuda_fail(err, "at_ensemble_create: cudaMalloc"); }
  char *base = (char *)e->scratch;
  e->d_members = (MemberParams *)base; base += up(b_members);
  e->d_order = (int32_t *)base; base += up(b_order);
  e->d_counter = (int32_t *)base; base += 256;
  e->d_member_stats = (double *)base; base += up(b_stats);
  e->d_member_diff = (double *)base; base += up(b_diff);
  e->d_summary = (double *)base; base += up(b_sum);
  // every member starts from Eq. "IC" with the analytic pre-history: ts-1 right-hand sides stored before step 0
  int64_t *d_first = (int64_t *)base;
  std::vector<int64_t> first(count);
  for (int r = 0; r < count; ++r) {
    first[r] = -(int64_t)(host[r].p.ts - 1);
    host[r].p.ab_first = d_first + r;
  }
  if ((err = cudaMemcpy(d_first, first.data(), b_first, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (err = cudaMemcpy(e->d_members, host.data(), b_members, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (err = cudaMemcpy(e->d_order, order.data(), b_order, cudaMemcpyHostToDevice)) != cudaSuccess) {
    cudaFree(e->scratch); delete e;
    return cuda_fail(err, "at_ensemble_create: upload");
  }
  int dev = 0, sms = 0, fit = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t dyn_smem = (size_t)(2 * max_nb + 15) / 16 * 16;
  if (dyn_smem > 48 * 1024) {
    delete e;
    return fail(AT_ERR_ARG, "at_ensemble_create: a member has too many PE sides");
  }
  e->dyn_smem = dyn_smem;
  int hmax = 1;
  bool any_ab = false, any_space = false;
  for (int r = 0; r < count; ++r) {
    hmax = std::max(hmax, (int)host[r].p.h);
    any_ab = any_ab || host[r].p.ts > 1;
    any_space = any_space || host[r].p.scheme >= AT_AT_SPACE2;
  }
  auto kernel = any_space ? ensemble_kernel<2, false, true>
                : hmax <= 2 ? (any_ab ? ensemble_kernel<2, true, false> : ensemble_kernel<2, false, false>)
                            : (any_ab ? ensemble_kernel<3, true, false> : ensemble_kernel<3, false, false>);
  if (any_space && (hmax > 2 || any_ab)) {
    // a mix of schemes expanded in space with order-6 or Adams-Bashforth members
    kernel = hmax <= 2 ? (any_ab ? ensemble_kernel<2, true, true> : ensemble_kernel<2, false, true>)
                       : (any_ab ? ensemble_kernel<3, true, true> : ensemble_kernel<3, false, true>);
  }
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kernel, threads, dyn_smem);
  if (ctas_per_sm <= 0) ctas_per_sm = fit;
  if (ctas_per_sm > fit) ctas_per_sm = fit;
  if (ctas_per_sm < 1) ctas_per_sm = 1;
  e->blocks = sms * ctas_per_sm;
  if (e->blocks > count) e->blocks = count;
  // capture: counter reset, persistent kernel, summary
  cudaStream_t cap;
  if ((err = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) {
    cudaFree(e->scratch); delete e;
    return cuda_fail(err, "at_ensemble_create: stream");
  }
  err = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (err == cudaSuccess) {
    reset_counter<<<1, 1, 0, cap>>>(e->d_counter);
    kernel<<<e->blocks, threads, e->dyn_smem, cap>>>(e->d_members, e->d_order, count, e->d_counter,
                                                    e->d_member_stats);
    twin_diff_kernel<<<count, 256, 0, cap>>>(e->d_members, e->d_member_diff);
    summary_kernel<<<1, 128, 0, cap>>>(e->d_member_stats, e->d_member_diff, e->d_members, count, e->ngroups,
                                       e->d_summary);
    err = cudaStreamEndCapture(cap, &e->graph);
  }
  if (err == cudaSuccess) err = cudaGraphInstantiate(&e->exec, e->graph, 0);
  cudaStreamDestroy(cap);
  if (err != cudaSuccess) {
    if (e->graph) cudaGraphDestroy(e->graph);
    cudaFree(e->scratch); delete e;
    return cuda_fail(err, "at_ensemble_create: graph");
  }
  *out = e;
  return AT_OK;
}

extern "C" int at_ensemble_run(at_ensemble_t *e) {
  if (!e) return fail(AT_ERR_ARG, "at_ensemble_run: NULL handle");
  cudaError_t err = cudaGraphLaunch(e->exec, e->stream);
  if (err != cudaSuccess) return cuda_fail(err, "at_ensemble_run");
  return AT_OK;
}

extern "C" int at_ensemble_stats(at_ensemble_t *e, at_stats_t *per_member, double *per_member_diff, int32_t cap,
                                 at_group_stats_t *groups, int32_t gcap, int32_t *ngroups) {
  if (!e || !ngroups) return fail(AT_ERR_ARG, "at_ensemble_stats: bad argument");
  std::vector<double> ms((size_t)e->count * kStatFields), md(2 * (size_t)e->count),
      sum(kGroupFields * (size_t)e->ngroups);
  cudaError_t err;
  if ((err = cudaMemcpyAsync(ms.data(), e->d_member_stats, ms.size() * sizeof(double), cudaMemcpyDeviceToHost,
                             e->stream)) != cudaSuccess ||
      (err = cudaMemcpyAsync(md.data(), e->d_member_diff, md.size() * sizeof(double), cudaMemcpyDeviceToHost,
                             e->stream)) != cudaSuccess ||
      (err = cudaMemcpyAsync(sum.data(), e->d_summary, sum.size() * sizeof(double), cudaMemcpyDeviceToHost,
                             e->stream)) != cudaSuccess ||
      (err = cudaStreamSynchronize(e->stream)) != cudaSuccess)
    return cuda_fail(err, "at_ensemble_stats");
  *ngroups = e->ngroups;
  for (int r = 0; r < e->count && r < cap; ++r) {
    if (per_member_diff) {
      per_member_diff[2 * r] = md[2 * r];
      per_member_diff[2 * r + 1] = md[2 * r + 1];
    }
    if (!per_member) continue;
    const double *s = &ms[(size_t)r * kStatFields];
    const double N = (double)e->member_n[r];
    at_stats_t &o = per_member[r];
    o.rms = std::sqrt(s[0] / N);
    o.max_abs = s[1];
    o.mean_abs = s[2] / N;
    o.mean = s[3] / N;
    o.rms_I = s[7] > 0 ? std::sqrt(s[4] / s[7]) : 0.0;
    o.rms_B = s[8] > 0 ? std::sqrt(s[5] / s[8]) : 0.0;
    o.ua_rms = std::sqrt(s[6] / N);
    o.n_I = (int64_t)s[7];
    o.n_B = (int64_t)s[8];
    o.step = e->member_steps[r];
  }
  for (int g = 0; groups && g < e->ngroups && g < gcap; ++g) {
    const double *o = &sum[kGroupFields * (size_t)g];
    at_group_stats_t &G = groups[g];
    G.key = e->group_key[g];
    G.count = (int32_t)o[2];
    G.ntwin = (int32_t)o[5];
    G.rms_mean = o[0];
    G.rms_var = o[1];
    G.abs_mean = o[8];
    G.diff_mean = o[3];
    G.diff_var = o[4];
    G.dabs_mean = o[6];
    G.dabs_var = o[7];
  }
  for (double v : ms)
    if (!std::isfinite(v)) return fail(AT_ERR_NONFINITE, "at_ensemble_stats: non-finite statistic");
  for (double v : md)
    if (!std::isfinite(v)) return fail(AT_ERR_NONFINITE, "at_ensemble_stats: non-finite twin difference");
  return AT_OK;
}

extern "C" int at_ensemble_destroy(at_ensemble_t *e) {
  if (!e) return AT_OK;
  cudaError_t err = cudaStreamSynchronize(e->stream);
  if (e->exec) cudaGraphExecDestroy(e->exec);
  if (e->graph) cudaGraphDestroy(e->graph);
  cudaFree(e->scratch);
  delete e;
  if (err != cudaSuccess) return cuda_fail(err, "at_ensemble_destroy");
  return AT_OK;
}
