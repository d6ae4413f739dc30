// fwd.cu -- the fused forward step of the asynchrony-tolerant (AT) scheme on sm_103a.
//
// One launch advances U^n -> U^{n+1} by forward Euler (Sec. 4.1, Eq. "time_disc" with one level):
//     U^{n+1}_i = U^n_i + dt sum_a ( -c_a D1_a U + alpha D2_a U )_i
// with the central differences and the AT tables folded into merged per-axis coefficients
//     s_{a,j} = dt ( -c_a cd1_j / dx_a + alpha cd2_j / dx_a^2 ),   s0 = 1 + sum_a s_{a,0},
// so an interior point costs one multiply and 2*h*dim fused multiply-adds.
//
// Points within h of a PE boundary (the set I_B of Sec. 2) read, for each stencil point across that
// boundary (a buffer point), the extrapolated halo value
//     u~ = sum_{m<T} w_m(k) U^{n-k-m}                                   (k = that side's delay)
// where w_m(k) are the stage-2 weights of Example 3.  Since sum_m w_m(k) CD(.. U^{n-k-m} ..) =
// CD(.. u~ ..) for the time-expanded tables ((1,2,2)b, (2,2,2)b, (1,4,2), (2,4,2)), the halo value is
// formed once and shared by the first- and second-derivative taps.  The delay k of every PE side is
// drawn in-kernel from Philox (Sec. 5.1) keyed by (seed, step, side) and clamped so that no level before
// 0 is read; one designated thread per side writes the raw draw to the delay log.
//
// The kernel is bound by the FP64 pipe on GB300 (2 FP64 FMA lanes per SM per clock nominal; about 1.6 per
// clock sustained for dependent FMA chains): each point costs the minimum 1 + 2 h dim FP64 operations, all of
// them FMAs -- the chain starts with fma(s0, u_i, +0) on a runtime zero, because a DMUL occupies the FP64
// pipe longer than a DFMA and the result is the same rounded product.
#include "stencil.cuh"

namespace {

using namespace atfd;

// 1D: each thread updates four consecutive points with 16-byte loads and stores.  A group that lies inside
// one PE, at least h from its edges and from the ends of the domain, takes the straight FMA path with four
// independent accumulation chains; any other group takes the general path point by point.
template <int H>
__global__ void __launch_bounds__(256) forward_1d_kernel(const StepParams p, const int64_t n_off, const int64_t *n_base) {
  const int64_t n = n_off + (n_base ? *n_base : 0);
  const double *__restrict__ un = p.ring + (n % p.R) * p.ntot;
  double *__restrict__ out = p.ring + ((n + 1) % p.R) * p.ntot;
  const int groups = (p.n[0] + 3) >> 2;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += gridDim.x * blockDim.x)
    group_1d<H, LdgNC>(p, un, out, n, g << 2);
}

// 3D: each thread updates four consecutive x points of one (y, z) row.  Rows y +- j and z +- j are read with
// the same 16-byte alignment (nx is a multiple of 4 on this path).
template <int H>
__global__ void __launch_bounds__(256) forward_3d_kernel(const StepParams p, const int64_t n_off, const int64_t *n_base) {
  const int64_t n = n_off + (n_base ? *n_base : 0);
  const double *__restrict__ un = p.ring + (n % p.R) * p.ntot;
  double *__restrict__ out = p.ring + ((n + 1) % p.R) * p.ntot;
  const int nx = p.n[0], ny = p.n[1], nz = p.n[2];
  const int gx = nx >> 2;
  const int64_t groups = (int64_t)gx * ny * nz;
  const int64_t sy = nx, sz = (int64_t)nx * ny;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = g / gx;
    const int x0 = (int)(g - row * gx) << 2;
    const int z = (int)(row / ny), y = (int)(row - (int64_t)z * ny);
    const int px = x0 % p.S[0], py = y % p.S[1], pz = z % p.S[2];
    const bool inx = (x0 >= 2) && (x0 + 6 <= nx) && (!p.use_pe[0] || (px >= H && px + 3 < p.S[0] - H));
    const bool iny = (y >= H) && (y + H < ny) && (!p.use_pe[1] || (py >= H && py < p.S[1] - H));
    const bool inz = (z >= H) && (z + H < nz) && (!p.use_pe[2] || (pz >= H && pz < p.S[2] - H));
    const int64_t i0 = row * nx + x0;
    if (inx && iny && inz) {
      const double2 a = LdgNC::ld2(un + i0 - 2), b = LdgNC::ld2(un + i0), c = LdgNC::ld2(un + i0 + 2), d = LdgNC::ld2(un + i0 + 4);
      const double v[8] = {a.x, a.y, b.x, b.y, c.x, c.y, d.x, d.y};
      double r[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) r[q] = axis_taps<H>(p.s[0], v + q + 2 - H, fma(p.s0, v[q + 2], p.zero));
#pragma unroll
      for (int ax = 1; ax < 3; ++ax) {
        const int64_t st = ax == 1 ? sy : sz;
#pragma unroll
        for (int j = -H; j <= H; ++j) {
          if (j == 0) continue;
          const double2 e = LdgNC::ld2(un + i0 + j * st), f = LdgNC::ld2(un + i0 + j * st + 2);
          r[0] = fma(p.s[ax][j + H], e.x, r[0]);
          r[1] = fma(p.s[ax][j + H], e.y, r[1]);
          r[2] = fma(p.s[ax][j + H], f.x, r[2]);
          r[3] = fma(p.s[ax][j + H], f.y, r[3]);
        }
      }
      reinterpret_cast<double2 *>(out + i0)[0] = make_double2(r[0], r[1]);
      reinterpret_cast<double2 *>(out + i0)[1] = make_double2(r[2], r[3]);
    } else {
      for (int q = 0; q < 4; ++q) {
        const int c[3] = {x0 + q, y, z};
        out[i0 + q] = point_update<3, H, LdgNC>(p, un, n, i0 + q, c);
      }
    }
  }
}

// Fallback for shapes the grouped kernels do not take (odd point counts, nx not a multiple of 4).
template <int DIM, int H>
__global__ void __launch_bounds__(256) forward_point_kernel(const StepParams p, const int64_t n_off, const int64_t *n_base) {
  const int64_t n = n_off + (n_base ? *n_base : 0);
  const double *__restrict__ un = p.ring + (n % p.R) * p.ntot;
  double *__restrict__ out = p.ring + ((n + 1) % p.R) * p.ntot;
  const int nx = p.n[0], ny = DIM == 3 ? p.n[1] : 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.ntot; i += (int64_t)gridDim.x * blockDim.x) {
    int c[3] = {(int)i, 0, 0};
    if (DIM == 3) {
      const int64_t yz = i / nx;
      c[0] = (int)(i - yz * nx);
      c[2] = (int)(yz / ny);
      c[1] = (int)(yz - (int64_t)c[2] * ny);
    }
    out[i] = point_update<DIM, H, LdgNC>(p, un, n, i, c);
  }
}

__global__ void add_steps_kernel(int64_t *n_base, int64_t v, int set) {
  if (set) *n_base = v; else *n_base += v;
}

}  // namespace

cudaError_t launch_step_counter(int64_t *n_base, int64_t v, bool set, cudaStream_t st) {
  add_steps_kernel<<<1, 1, 0, st>>>(n_base, v, set ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_forward_step(const StepParams &p, int64_t n, const int64_t *n_base, cudaStream_t st) {
  const int threads = 256;
  const int max_blocks = 152 * 8 * 4;
  auto grid = [&](int64_t work) { int64_t b = (work + threads - 1) / threads; return (int)(b < max_blocks ? b : max_blocks); };
  const bool even = (p.ntot % 2) == 0 && (reinterpret_cast<uintptr_t>(p.ring) % 16) == 0;
  if (p.dim == 1) {
    if (even) {
      const int64_t groups = (p.ntot + 3) / 4;
      if (p.h == 1) forward_1d_kernel<1><<<grid(groups), threads, 0, st>>>(p, n, n_base);
      else forward_1d_kernel<2><<<grid(groups), threads, 0, st>>>(p, n, n_base);
    } else {
      if (p.h == 1) forward_point_kernel<1, 1><<<grid(p.ntot), threads, 0, st>>>(p, n, n_base);
      else forward_point_kernel<1, 2><<<grid(p.ntot), threads, 0, st>>>(p, n, n_base);
    }
  } else {
    if (p.n[0] % 4 == 0 && even) {
      const int64_t groups = p.ntot / 4;
      if (p.h == 1) forward_3d_kernel<1><<<grid(groups), threads, 0, st>>>(p, n, n_base);
      else forward_3d_kernel<2><<<grid(groups), threads, 0, st>>>(p, n, n_base);
    } else {
      if (p.h == 1) forward_point_kernel<3, 1><<<grid(p.ntot), threads, 0, st>>>(p, n, n_base);
      else forward_point_kernel<3, 2><<<grid(p.ntot), threads, 0, st>>>(p, n, n_base);
    }
  }
  return cudaGetLastError();
}
