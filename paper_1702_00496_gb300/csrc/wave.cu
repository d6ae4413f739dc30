// wave.cu -- multi-sine fields and error statistics (arXiv:1702.00496, Sec. 5.1 and Sec. 4).
//
//  launch_wave_field   u(x, t) = prod_axes sum_kappa A exp(-alpha kappa^2 t) sin(kappa (x_a - c_a t) + phi)
//                      -- Eq. "IC" at t = 0 and Eq. "ana_sol" (travelling phase kappa (x - c t)) for t > 0.
//                      In 3D the per-axis sums are tabulated first (n0+n1+n2 values) and multiplied.
//  launch_error_stats  E = U - u_a and its averages over I, I_I, I_B (Sec. 4): sum E^2, max |E|, sum |E|,
//                      sum E, sum E^2 on I_I and I_B, sum u_a^2, |I_I|, |I_B|.  Fixed grid of
//                      AT_STAT_BLOCKS blocks, per-block partials, then one block reduces them in a fixed
//                      order, so the result is deterministic.
#include <cmath>
#include <utility>

#include "internal.h"
#include "modes.cuh"

namespace {

// Sum over the modes of axis a at grid point i, for the time t of the launch (w.amp holds A exp(-alpha kappa^2 t),
// scaled on the host): the three-term recurrences for integer wavenumbers, else a sine per mode.
__device__ __forceinline__ double axis_sum(const WaveParams &w, int a, int i, double t) {
  if (w.ms[a].rot) return atfd::mode_sum(w.ms[a], w.nmodes, (double)i * w.xpi[a]);
  const double x = (double)i * w.dx[a];
  const double shift = w.c[a] * t;
  double s = 0.0;
  for (int q = 0; q < w.nmodes; ++q) s += w.amp[a][q] * sin(w.kappa[a][q] * (x - shift) + w.phase[a][q]);
  return s;
}

WaveParams at_time(const WaveParams &w0, double t) {
  WaveParams w = w0;
  for (int a = 0; a < 3; ++a) {
    if (a < w.dim) fill_modes(&w.ms[a], w0.amp[a], w0.phase[a], w0.kappa[a], w.nmodes, w0.alpha, w0.c[a], t);
    else w.ms[a].rot = 0;
  }
  for (int a = 0; a < w.dim; ++a)
    for (int q = 0; q < w.nmodes; ++q)
      if (t != 0.0) w.amp[a][q] = w0.amp[a][q] * std::exp(-w0.alpha * w0.kappa[a][q] * w0.kappa[a][q] * t);
  return w;
}

__global__ void axis_table_kernel(const WaveParams w, double t, double *tables) {
  const int total = w.n[0] + w.n[1] + w.n[2];
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    int a = 0, i = g;
    while (a < 2 && i >= w.n[a]) { i -= w.n[a]; ++a; }
    tables[g] = a < w.dim ? axis_sum(w, a, i, t) : 1.0;
  }
}

__global__ void field_1d_kernel(const WaveParams w, double t, double *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < w.n[0]; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = axis_sum(w, 0, (int)i, t);
}

__global__ void field_3d_kernel(const WaveParams w, const double *tables, double *out) {
  const int64_t nx = w.n[0], ny = w.n[1], ntot = nx * ny * w.n[2];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ntot; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t yz = i / nx;
    const int x = (int)(i - yz * nx), z = (int)(yz / ny), y = (int)(yz - z * ny);
    out[i] = tables[x] * tables[w.n[0] + y] * tables[w.n[0] + w.n[1] + z];
  }
}

// REF = false: E = U - u_a with u_a the analytic solution at time t; REF = true: E = U - V with V a reference field
// `refine` times finer on every axis, sampled at the coarse points (V at (refine x, refine y, refine z)).
template <int DIM, bool REF>
__global__ void __launch_bounds__(256) stats_partial_kernel(const WaveParams w, const StepParams p, const double *u,
                                                            double t, const double *tables, double *partials,
                                                            const double *ref, int refine) {
  double acc[AT_STAT_FIELDS];
#pragma unroll
  for (int f = 0; f < AT_STAT_FIELDS; ++f) acc[f] = 0.0;
  const int64_t nx = w.n[0], ny = w.n[1];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.ntot; i += (int64_t)gridDim.x * blockDim.x) {
    int c[3] = {(int)i, 0, 0};
    if (DIM == 3) {
      const int64_t yz = i / nx;
      c[0] = (int)(i - yz * nx); c[2] = (int)(yz / ny); c[1] = (int)(yz - (int64_t)c[2] * ny);
    }
    double ua;
    if (REF) {
      const int64_t nxf = nx * refine, nyf = ny * refine;
      ua = ref[((int64_t)c[2] * refine * nyf + (int64_t)c[1] * refine) * nxf + (int64_t)c[0] * refine];
    } else if (DIM == 1) {
      ua = axis_sum(w, 0, c[0], t);
    } else {
      ua = tables[c[0]] * tables[w.n[0] + c[1]] * tables[w.n[0] + w.n[1] + c[2]];
    }
    bool inB = false;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int pos = c[a] % p.S[a];
      if (p.use_pe[a] && (pos < p.h || pos >= p.S[a] - p.h)) inB = true;
    }
    const double e = u[i] - ua;
    acc[0] += e * e;
    acc[1] = fmax(acc[1], fabs(e));
    acc[2] += fabs(e);
    acc[3] += e;
    if (inB) { acc[5] += e * e; acc[8] += 1.0; } else { acc[4] += e * e; acc[7] += 1.0; }
    acc[6] += ua * ua;
    if (e != e) acc[1] = e;  // keep a NaN visible through the max
  }
  __shared__ double red[AT_STAT_FIELDS][256];
#pragma unroll
  for (int f = 0; f < AT_STAT_FIELDS; ++f) red[f][threadIdx.x] = acc[f];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
#pragma unroll
      for (int f = 0; f < AT_STAT_FIELDS; ++f) {
        const double o = red[f][threadIdx.x + s];
        red[f][threadIdx.x] = (f == 1) ? ((o != o) ? o : fmax(red[f][threadIdx.x], o)) : red[f][threadIdx.x] + o;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < AT_STAT_FIELDS) partials[(int64_t)blockIdx.x * AT_STAT_FIELDS + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void __launch_bounds__(AT_STAT_BLOCKS) stats_final_kernel(const double *partials, double *result) {
  __shared__ double red[AT_STAT_BLOCKS];
  for (int f = 0; f < AT_STAT_FIELDS; ++f) {
    red[threadIdx.x] = partials[(int64_t)threadIdx.x * AT_STAT_FIELDS + f];
    __syncthreads();
    for (int s = AT_STAT_BLOCKS / 2; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s) {
        const double o = red[threadIdx.x + s];
        red[threadIdx.x] = (f == 1) ? ((o != o) ? o : fmax(red[threadIdx.x], o)) : red[threadIdx.x] + o;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) result[f] = red[0];
    __syncthreads();
  }
}

}  // namespace

void fill_modes(ModeSet *ms, const double *amp, const double *phase, const double *kappa, int nmodes, double alpha,
                double c, double t) {
  int idx[AT_MAX_MODES];
  bool ok = nmodes >= 1 && nmodes <= AT_MAX_MODES;
  for (int q = 0; ok && q < nmodes; ++q) {
    idx[q] = q;
    ok = kappa[q] >= 1.0 && kappa[q] <= (double)AT_MAX_KROT && kappa[q] == std::floor(kappa[q]);
  }
  ms->rot = ok ? 1 : 0;
  ms->kmax = 0;
  if (!ok) return;
  for (int q = 1; q < nmodes; ++q)  // insertion sort of the modes by wavenumber (stable)
    for (int r = q; r > 0 && kappa[idx[r - 1]] > kappa[idx[r]]; --r) std::swap(idx[r - 1], idx[r]);
  for (int q = 0; q < nmodes; ++q) {
    const int m = idx[q];
    const double k = kappa[m];
    const double A = t != 0.0 ? amp[m] * std::exp(-alpha * k * k * t) : amp[m];
    const double ph = phase[m] - k * c * t;
    ms->kr[q] = (int32_t)k;
    ms->ac[q] = A * std::cos(ph);
    ms->as[q] = A * std::sin(ph);
    if ((int32_t)k > ms->kmax) ms->kmax = (int32_t)k;
  }
}

cudaError_t launch_wave_field(const WaveParams &w0, double t, double *tables, double *out, cudaStream_t st) {
  const WaveParams w = at_time(w0, t);
  if (w.dim == 1) {
    const int64_t blocks = (w.n[0] + 255) / 256;
    field_1d_kernel<<<(int)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, st>>>(w, t, out);
  } else {
    axis_table_kernel<<<8, 256, 0, st>>>(w, t, tables);
    const int64_t ntot = (int64_t)w.n[0] * w.n[1] * w.n[2];
    const int64_t blocks = (ntot + 255) / 256;
    field_3d_kernel<<<(int)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, st>>>(w, tables, out);
  }
  return cudaGetLastError();
}

cudaError_t launch_error_stats(const WaveParams &w0, const StepParams &p, const double *u, double t, double *tables,
                               double *partials, double *result, cudaStream_t st) {
  const WaveParams w = at_time(w0, t);
  if (w.dim == 1) {
    stats_partial_kernel<1, false><<<AT_STAT_BLOCKS, 256, 0, st>>>(w, p, u, t, tables, partials, nullptr, 1);
  } else {
    axis_table_kernel<<<8, 256, 0, st>>>(w, t, tables);
    stats_partial_kernel<3, false><<<AT_STAT_BLOCKS, 256, 0, st>>>(w, p, u, t, tables, partials, nullptr, 1);
  }
  stats_final_kernel<<<1, AT_STAT_BLOCKS, 0, st>>>(partials, result);
  return cudaGetLastError();
}

cudaError_t launch_error_stats_ref(const WaveParams &w, const StepParams &p, const double *u, const double *ref,
                                   int refine, double *partials, double *result, cudaStream_t st) {
  if (w.dim == 1)
    stats_partial_kernel<1, true><<<AT_STAT_BLOCKS, 256, 0, st>>>(w, p, u, 0.0, nullptr, partials, ref, refine);
  else
    stats_partial_kernel<3, true><<<AT_STAT_BLOCKS, 256, 0, st>>>(w, p, u, 0.0, nullptr, partials, ref, refine);
  stats_final_kernel<<<1, AT_STAT_BLOCKS, 0, st>>>(partials, result);
  return cudaGetLastError();
}
