// fwd.cu -- the fused forward step of the asynchrony-tolerant (AT) scheme on sm_103a.
//
// One launch advances U^n -> U^{n+1} by forward Euler (Sec. 4.1, Eq. "time_disc" with one level):
//     U^{n+1}_i = U^n_i + dt sum_a ( -c_a D1_a U + alpha D2_a U )_i = U^n_i + dt f^n_i
// with the central differences and the AT tables folded into merged per-axis coefficients
//     s_{a,j} = dt ( -c_a cd1_j / dx_a + alpha cd2_j / dx_a^2 ),   s0 = 1 + sum_a s_{a,0},
// so an interior point costs one multiply and 2*h*dim fused multiply-adds.  With two or three time levels
// (Adams-Bashforth, Eq. "time_disc"; Eq. "time_ab2") the chain, with s0 lacking the 1, forms dt f^n; the launch
// adds the stored dt f^{n-1}, dt f^{n-2} of the previous launches with their weights and stores dt f^n.
//
// Points within h of a PE boundary (the set I_B of Sec. 2) read, for each stencil point across that
// boundary (a buffer point), the extrapolated halo value
//     u~ = sum_{m<T} w_m(k) U^{n-k-m}                                   (k = that side's delay)
// where w_m(k) are the stage-2 weights of Example 3.  Since sum_m w_m(k) CD(.. U^{n-k-m} ..) =
// CD(.. u~ ..) for the time-expanded tables ((1,2,2)b, (2,2,2)b, (1,4,2), (2,4,2), (2,6,2)), the halo value is
// formed once and shared by the first- and second-derivative taps.  The delay k of every PE side is
// drawn from Philox (Sec. 5.1) keyed by (seed, step, side) once per step -- by the launch of the previous
// step, into a double-buffered array -- and clamped so that no level before 0 is read.
//
// The kernel is bound by the FP64 pipe on GB300 (2 FP64 FMA lanes per SM per clock nominal; about 1.6 per
// clock sustained for dependent FMA chains): each point costs the minimum 1 + 2 h dim FP64 operations, all of
// them FMAs -- the chain starts with fma(s0, u_i, +0) on a runtime zero, because a DMUL occupies the FP64
// pipe longer than a DFMA and the result is the same rounded product.
#include <algorithm>
#include <cstring>

#include "stencil.cuh"

namespace {

using namespace atfd;

// Grouped kernel: a thread updates four consecutive x points per iteration (grid-stride); every thread
// also draws the delays of one slice of the PE sides for step n+1 into the other half of the double-buffered
// delay array, so the next launch finds them ready.
template <int DIM, int H, int AB, int KIND>
__global__ void __launch_bounds__(512) forward_group_kernel(const StepParams p, const int64_t n_off,
                                                            const int64_t *n_base) {
  const int64_t n = n_off + (n_base ? *n_base : 0);
  const double *__restrict__ un = p.ring + (n % p.R) * p.ntot;
  double *__restrict__ out = p.ring + ((n + 1) % p.R) * p.ntot;
  const uint8_t *keff = p.keff + (n & 1) * p.nb;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nthreads = (int64_t)gridDim.x * blockDim.x;
  draw_sides(p, n + 1, tid, nthreads, p.keff + ((n + 1) & 1) * p.nb);
  const int gx = p.n[0] >> 2;
  const int64_t groups = (int64_t)gx * p.n[1] * p.n[2];
  for (int64_t k = tid; k < groups; k += nthreads) {
    if (DIM == 1) {
      const int64_t g = group_1d_order(p, k);
      group_step<1, H, LdgNC, AB, KIND>(p, keff, un, out, n, (int)(g << 2), 0, 0);
    } else {
      const int64_t g = p.order ? (int64_t)p.order[k] : k;
      const int64_t r = g / gx;
      const int x0 = (int)(g - r * gx) << 2;
      const int z = (int)(r / p.n[1]), y = (int)(r - (int64_t)z * p.n[1]);
      group_step<3, H, LdgNC, AB, KIND>(p, keff, un, out, n, x0, y, z);
    }
  }
}

// Blocks of K steps (1D forward Euler, central and time-expanded rows).  Away from PE boundaries the step is the
// same linear stencil at every point and step, so K steps of it are one stencil of half-width h K: its taps ck are
// the K-fold composition of the merged taps, and a group whose K-step stencil stays inside its PE gets U^{n+K}
// from U^n with 2 h K + 1 FMAs per point instead of K (2 h + 1).  The cells near a PE boundary, whose buffer points
// take the delayed halo values of every step, are advanced step by step: the zone launch runs steps n .. n+K-2 of
// the step kernel's arithmetic on the cells within zr[j] of each boundary (zones that shrink by at least h per
// step), and the block launch gives the edge groups their last step from U^{n+K-1}.  The zones hold the face
// strips, so the intermediate levels are in the ring wherever a later step reads a delayed level.  The delays of
// steps n+1 .. n+K-1 are drawn by the zone launch and the delays of step n+K by the block launch, so the delay log
// and the effective delays are those of single steps.

// Zone launch of the block starting at step n: a warp per PE boundary runs steps n .. n+K-2 on its zone.  A zone
// lies within S/2 of its boundary, so its cells read across that boundary only: the warp draws the delays of the two
// sides facing it (the right side of the PE before, the left side of the PE after) for steps n+1 .. n+K-1 itself,
// into the effective-delay buffer (whose slot for each step and side only this warp uses) and the log, and the
// steps are separated by __syncwarp, so the loads are coherent ones.  A zone group reads only the delay of the side
// it reaches across (its own), never one that another warp may be writing.  Without PE boundaries warp 0 only draws.
template <int H, int K>
__global__ void __launch_bounds__(128) forward_zones_kernel(const StepParams p, const int64_t n_off,
                                                            const int64_t *n_base) {
  // the block launch that follows may start now: its inner groups read only U^n, and it waits for this grid before
  // its edge groups and its delay draws
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  // Each warp holds its boundary's region -- cells b - RR .. b + RR - 1, RR = zr[0] + h -- at levels n .. n+K-1 in
  // shared memory: U^n is read once, each step's zone is computed from the level before it there, and only levels
  // before n (the delayed halo levels at the face strips) are read from the ring.  The arithmetic is the step
  // kernel's: the centre tap, then the taps in offset order, a buffer point's value extrapolated over the delayed
  // levels w_m(k) in the order m = 0 .. T-1.
  constexpr int CELLS = 64;  // 2 RR <= 2 (zr[0] + h) <= 54 for h <= 3, K <= 4
  __shared__ double lev[4][K][CELLS];
  const int64_t n = n_off + (n_base ? *n_base : 0);
  const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t P = p.pe[0], nbound = p.use_pe[0] ? P : 0;
  const int nx = p.n[0], RR = p.zr[0] + H;
  for (int64_t b = warp; b < (nbound > 0 ? nbound : 1); b += nwarps) {
    const int64_t sides[2] = {nbound ? 2 * ((b + P - 1) % P) + 1 : 0, nbound ? 2 * b : 1};
    const int base = (int)(b * p.S[0]) - RR;  // cell of local index 0 (before wrapping)
    if (nbound)
      for (int i = lane; i < 2 * RR; i += 32) lev[wb][0][i] = p.ring[(n % p.R) * p.ntot + wrap_coord(base + i, nx)];
    __syncwarp();
    for (int j = 0; j + 1 < K; ++j) {
      const int64_t st = n + j;  // the step this pass computes; it draws the delays of step st + 1
      const uint8_t *keff = p.keff + (st & 1) * p.nb;
      // delays of step st seen across this boundary: by the cells left of it (the right side of the PE before) and
      // by the cells right of it (the left side of the PE after); read before this pass's draw of step st + 1
      const int k_lo = nbound ? keff[sides[0]] : 0, k_hi = nbound ? keff[sides[1]] : 0;
      __syncwarp();
      if (lane < 2) {
        const int64_t side = sides[lane];
        int raw = 0;
        if (p.scheme != 0)
          raw = delay_draw(p.seed, (uint32_t)(st + 1), (uint32_t)side, p.L, p.use_thr ? p.thr : nullptr);
        p.keff[((st + 1) & 1) * p.nb + side] = (uint8_t)delay_clamp(raw, st + 1, p.T);
        if (p.log != nullptr && st + 1 < p.log_steps) p.log[(st + 1) * p.nb + side] = (uint8_t)raw;
      }
      if (nbound) {
        double *out = p.ring + ((st + 1) % p.R) * p.ntot;
        const int r = p.zr[j];
        for (int i = RR - r + lane; i < RR + r; i += 32) {
          const bool left = i < RR;
          double acc = fma(p.s0, lev[wb][j][i], p.zero);
#pragma unroll
          for (int t = -H; t <= H; ++t) {
            if (t == 0) continue;
            const int ii = i + t;
            double v = lev[wb][j][ii];
            const int k = left == (ii < RR) ? 0 : (left ? k_lo : k_hi);  // a tap across the boundary: buffer point
            if (k > 0) {
              const int cell = wrap_coord(base + ii, nx);
              double h = 0.0;
#pragma unroll
              for (int m = 0; m < AT_MAX_T; ++m) {
                if (m >= p.T) break;
                const int64_t q = st - k - m;  // level read: in shared memory from n on, else in the ring
                const double u = q >= n ? lev[wb][q - n][ii] : p.ring[(q % p.R) * p.ntot + cell];
                h = m == 0 ? fma(p.w[k][0], u, p.zero) : fma(p.w[k][m], u, h);
              }
              v = h;
            }
            acc = fma(p.s[0][t + H], v, acc);
          }
          lev[wb][j + 1][i] = acc;
          out[wrap_coord(base + i, nx)] = acc;
        }
      }
      __syncwarp();
    }
  }
}

// The last step m = n + K - 1 of a block: inner groups U^{n+K} = ck * U^n, edge groups the step from U^m.
template <int H, int K>
__global__ void __launch_bounds__(512) forward_block_kernel(const StepParams p, const int64_t n_off,
                                                            const int64_t *n_base) {
  constexpr int TK = H * K;                  // half-width of the composed stencil
  constexpr int WK = (TK + 1) / 2 * 2;       // its x window, rounded to even cells (16-byte loads)
  constexpr int NW = 4 + 2 * WK;
  const int64_t m = n_off + (n_base ? *n_base : 0), n0 = m - (K - 1);
  const double *__restrict__ u0 = p.ring + (n0 % p.R) * p.ntot;
  const double *__restrict__ um = p.ring + (m % p.R) * p.ntot;
  double *__restrict__ out = p.ring + ((m + 1) % p.R) * p.ntot;
  const uint8_t *keff = p.keff + (m & 1) * p.nb;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nthreads = (int64_t)gridDim.x * blockDim.x;
  const int nx = p.n[0];
  const int64_t groups = nx >> 2;
  const int64_t gS = p.use_pe[0] ? p.S[0] >> 2 : groups;
  const int64_t n_inner = (groups / gS) * (gS - 2 * p.fe);
  // Inner groups first: they read U^n only, so they may run while the zone launch (this block's steps n .. m-1 near
  // the PE boundaries, launched with a programmatic dependency) still does.  Then wait for it: the edge groups read
  // its U^m, and the delays of step m+1 go into the buffer slot its first step reads.
  for (int64_t k = tid; k < n_inner; k += nthreads) {
    const int x0 = (int)(group_1d_order_e(p, k, p.fe) << 2);
    double v[NW];
    if (x0 >= WK && x0 + 4 + WK <= nx) {
#pragma unroll
      for (int t = 0; t < NW; t += 2) {
        const double2 a = LdgNC::ld2(u0 + x0 - WK + t);
        v[t] = a.x; v[t + 1] = a.y;
      }
    } else {
#pragma unroll
      for (int t = 0; t < NW; ++t) v[t] = LdgNC::ld(u0 + wrap_coord(x0 - WK + t, nx));
    }
    double r[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double acc = fma(p.ck[TK], v[q + WK], p.zero);
#pragma unroll
      for (int j = -TK; j <= TK; ++j)
        if (j != 0) acc = fma(p.ck[j + TK], v[q + WK + j], acc);
      r[q] = acc;
    }
    reinterpret_cast<double2 *>(out + x0)[0] = make_double2(r[0], r[1]);
    reinterpret_cast<double2 *>(out + x0)[1] = make_double2(r[2], r[3]);
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  draw_sides(p, m + 1, tid, nthreads, p.keff + ((m + 1) & 1) * p.nb);
  for (int64_t k = n_inner + tid; k < groups; k += nthreads)
    group_step<1, H, LdgNC, false, 0>(p, keff, um, out, m, (int)(group_1d_order_e(p, k, p.fe) << 2), 0, 0);
}

__device__ __forceinline__ void point_coords(const StepParams &p, int dim, int64_t i, int c[3]) {
  c[0] = (int)i; c[1] = 0; c[2] = 0;
  if (dim == 3) {
    const int nx = p.n[0], ny = p.n[1];
    const int64_t yz = i / nx;
    c[0] = (int)(i - yz * nx);
    c[2] = (int)(yz / ny);
    c[1] = (int)(yz - (int64_t)c[2] * ny);
  }
}

// Fallback for shapes the grouped kernel does not take (n[0] not a multiple of 4, odd slots).
template <int DIM, int H, bool AB, int KIND>
__global__ void __launch_bounds__(512) forward_point_kernel(const StepParams p, const int64_t n_off,
                                                            const int64_t *n_base) {
  const int64_t n = n_off + (n_base ? *n_base : 0);
  const double *__restrict__ un = p.ring + (n % p.R) * p.ntot;
  double *__restrict__ out = p.ring + ((n + 1) % p.R) * p.ntot;
  const uint8_t *keff = p.keff + (n & 1) * p.nb;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nthreads = (int64_t)gridDim.x * blockDim.x;
  draw_sides(p, n + 1, tid, nthreads, p.keff + ((n + 1) & 1) * p.nb);
  for (int64_t i = tid; i < p.ntot; i += nthreads) {
    int c[3];
    point_coords(p, DIM, i, c);
    if (DIM == 1 && KIND == 1) {
      double r[1] = {point_update_burgers<H, LdgNC>(p, keff, un, n, i)};
      const double u[1] = {un[i]};
      if (AB) ab_combine<1>(p, n, i, u, r);
      else r[0] = u[0] + r[0];
      out[i] = r[0];
      continue;
    }
    double r[1] = {(KIND == 2 && H == 1) ? point_update_space<DIM, LdgNC>(p, keff, un, n, i, c)
                                         : point_update<DIM, H, LdgNC>(p, keff, un, n, i, c)};
    if (AB) {
      const double u[1] = {un[i]};
      ab_combine<1>(p, n, i, u, r);
    }
    out[i] = r[0];
  }
}

// dt f(u) with central differences everywhere (p carries no PE split and s0 without the 1): the right-hand
// sides before the first step of an Adams-Bashforth run.
template <int DIM, int H>
__global__ void __launch_bounds__(256) sync_rhs_kernel(const StepParams p, const double *__restrict__ u,
                                                       double *__restrict__ out, int grouped) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nthreads = (int64_t)gridDim.x * blockDim.x;
  if (grouped) {
    const int gx = p.n[0] >> 2;
    for (int64_t g = tid; g < p.ntot / 4; g += nthreads) {
      const int64_t r = g / gx;
      const int x0 = (int)(g - r * gx) << 2;
      const int z = (int)(r / p.n[1]), y = (int)(r - (int64_t)z * p.n[1]);
      double f[4], uc[4];
      group_eval<DIM, H, LdgNC, false>(p, p.keff, u, 0, x0, y, z, f, uc);
      const int64_t i0 = (DIM == 3 ? ((int64_t)z * p.n[1] + y) * p.n[0] : 0) + x0;
      for (int q = 0; q < 4; ++q) out[i0 + q] = f[q];
    }
  } else {
    for (int64_t i = tid; i < p.ntot; i += nthreads) {
      int c[3];
      point_coords(p, DIM, i, c);
      out[i] = point_update<DIM, H, LdgNC>(p, p.keff, u, 0, i, c);
    }
  }
}

__global__ void draw_first_kernel(const StepParams p, int64_t n) {
  draw_sides(p, n, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x,
             p.keff + (n & 1) * p.nb);
}

__global__ void add_steps_kernel(int64_t *n_base, int64_t v, int set) {
  if (set) *n_base = v; else *n_base += v;
}

}  // namespace

cudaError_t launch_step_counter(int64_t *n_base, int64_t v, bool set, cudaStream_t st) {
  add_steps_kernel<<<1, 1, 0, st>>>(n_base, v, set ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_draw_delays(const StepParams &p, int64_t n, cudaStream_t st) {
  const int64_t blocks = (p.nb + 255) / 256;
  draw_first_kernel<<<(int)(blocks < 1024 ? blocks : 1024), 256, 0, st>>>(p, n);
  return cudaGetLastError();
}

namespace {

// groups of four x points must not straddle a PE and must start on 16 bytes
bool grouped_shape(const StepParams &p, const void *base) {
  return p.n[0] % 4 == 0 && (!p.use_pe[0] || p.S[0] % 4 == 0) && (reinterpret_cast<uintptr_t>(base) % 16) == 0 &&
         (p.frhs == nullptr || (reinterpret_cast<uintptr_t>(p.frhs) % 16) == 0);
}

// AB: 0 forward Euler, 1 Adams-Bashforth, 2 AB2 with both levels stored (the 1D linear grouped step only; Burgers'
// step, 3D and the per-point fallback take the general form: Burgers' AB2 step measured 462 against 406 us in it).
template <int DIM, int H, int AB>
void launch_typed(const StepParams &p, bool grouped, int blocks, int threads, int64_t n, const int64_t *n_base,
                  cudaStream_t st) {
  constexpr int ABG = AB ? 1 : 0;
  if (DIM == 1 && p.burgers) {
    if (grouped) forward_group_kernel<1, H, ABG, 1><<<blocks, threads, 0, st>>>(p, n, n_base);
    else forward_point_kernel<1, H, ABG != 0, 1><<<blocks, threads, 0, st>>>(p, n, n_base);
    return;
  }
  if constexpr (H == 1 && !AB) {
    if (p.scheme >= AT_AT_SPACE2) {  // rows expanded in space: order 2, forward Euler only
      if (grouped) forward_group_kernel<DIM, 1, false, 2><<<blocks, threads, 0, st>>>(p, n, n_base);
      else forward_point_kernel<DIM, 1, false, 2><<<blocks, threads, 0, st>>>(p, n, n_base);
      return;
    }
  }
  if (grouped) forward_group_kernel<DIM, H, DIM == 1 ? AB : ABG, 0><<<blocks, threads, 0, st>>>(p, n, n_base);
  else forward_point_kernel<DIM, H, AB != 0, 0><<<blocks, threads, 0, st>>>(p, n, n_base);
}

template <int DIM, int AB>
void launch_h(const StepParams &p, bool grouped, int blocks, int threads, int64_t n, const int64_t *n_base,
              cudaStream_t st) {
  if (p.h == 1) launch_typed<DIM, 1, AB>(p, grouped, blocks, threads, n, n_base, st);
  else if (p.h == 2) launch_typed<DIM, 2, AB>(p, grouped, blocks, threads, n, n_base, st);
  else launch_typed<DIM, 3, AB>(p, grouped, blocks, threads, n, n_base, st);
}

int sm_count() {
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

}  // namespace

cudaError_t launch_forward_step(const StepParams &p, int64_t n, const int64_t *n_base, cudaStream_t st) {
  const int threads = p.threads > 0 ? p.threads : 256;
  const int max_blocks = sm_count() * (p.blocks_per_sm > 0 ? p.blocks_per_sm : 32);
  const bool grouped = grouped_shape(p, p.ring);
  const int64_t work = grouped ? p.ntot / 4 : p.ntot;
  const int64_t b = (work + threads - 1) / threads;
  const int blocks = (int)(b < max_blocks ? b : max_blocks);
  // a launch inside a captured graph (n_base set) runs only at steps at or after ab_steady
  const bool ab = p.ts > 1, steady = p.ts == 2 && (n_base != nullptr || n >= p.ab_steady);
  if (p.dim == 1) {
    if (steady) launch_h<1, 2>(p, grouped, blocks, threads, n, n_base, st);
    else if (ab) launch_h<1, 1>(p, grouped, blocks, threads, n, n_base, st);
    else launch_h<1, 0>(p, grouped, blocks, threads, n, n_base, st);
  } else {
    if (ab) launch_h<3, 1>(p, grouped, blocks, threads, n, n_base, st);
    else launch_h<3, 0>(p, grouped, blocks, threads, n, n_base, st);
  }
  return cudaGetLastError();
}

namespace {

template <int H, int K>
void launch_block_typed(const StepParams &p, int blocks, int zblocks, int threads, int64_t n_off,
                        const int64_t *n_base, cudaStream_t st) {
  forward_zones_kernel<H, K><<<zblocks, 128, 0, st>>>(p, n_off, n_base);
  // the block launch depends programmatically on the zone launch (it waits for it inside, before its edge groups)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, forward_block_kernel<H, K>, p, n_off + K - 1, n_base);
}

template <int H>
void launch_block_h(const StepParams &p, int blocks, int zblocks, int threads, int64_t n_off, const int64_t *n_base,
                    cudaStream_t st) {
  if (p.fuse_k == 2) launch_block_typed<H, 2>(p, blocks, zblocks, threads, n_off, n_base, st);
  else if (p.fuse_k == 3) launch_block_typed<H, 3>(p, blocks, zblocks, threads, n_off, n_base, st);
  else launch_block_typed<H, 4>(p, blocks, zblocks, threads, n_off, n_base, st);
}

}  // namespace

cudaError_t launch_forward_block(const StepParams &p, int64_t n_off, const int64_t *n_base, cudaStream_t st) {
  const int threads = p.threads > 0 ? p.threads : 256;
  const int max_blocks = sm_count() * (p.blocks_per_sm > 0 ? p.blocks_per_sm : 32);
  const int64_t b = (p.ntot / 4 + threads - 1) / threads;
  const int blocks = (int)(b < max_blocks ? b : max_blocks);
  const int64_t nwarps = p.use_pe[0] ? p.pe[0] : 1;  // zone launch: one warp per PE boundary, four per block
  const int64_t zb = (nwarps + 3) / 4;
  const int zblocks = (int)(zb < max_blocks ? zb : max_blocks);
  if (p.h == 1) launch_block_h<1>(p, blocks, zblocks, threads, n_off, n_base, st);
  else if (p.h == 2) launch_block_h<2>(p, blocks, zblocks, threads, n_off, n_base, st);
  else launch_block_h<3>(p, blocks, zblocks, threads, n_off, n_base, st);
  return cudaGetLastError();
}

// Zone radii of a K-step block: the edge groups of the last step reach 4 ceil(h K / 4) cells in from each PE end and
// read U^{n+K-1} h cells further; each earlier step's zone reaches h cells further than the next one's (multiples
// of 4, so zones are whole groups).
static void fuse_radii(int h, int K, int *fe, int zr[]) {
  const int reach = (h * K + 3) / 4 * 4;
  *fe = reach / 4;
  int r = reach;
  for (int j = K - 2; j >= 0; --j) {
    r = (r + h + 3) / 4 * 4;
    zr[j] = r;
  }
}

int fuse_max_k(const StepParams &p, const void *ring, int kmax) {
  if (p.dim != 1 || p.scheme > AT_AT || p.burgers || p.ts != 1 || !grouped_shape(p, ring)) return 1;
  for (int K = kmax < AT_MAX_FUSE ? kmax : AT_MAX_FUSE; K >= 2; --K) {
    if (p.R <= K) continue;  // U^n must stay in the ring while U^{n+K} is written
    int fe, zr[AT_MAX_FUSE];
    fuse_radii(p.h, K, &fe, zr);
    const int WK = (p.h * K + 1) / 2 * 2;
    if (p.n[0] < 2 * (4 + 2 * WK)) continue;  // the composed window stays within one wrap of the domain
    if (p.use_pe[0] && (2 * zr[0] > p.S[0] || p.S[0] / 4 <= 2 * fe)) continue;
    if (p.use_pe[0]) {  // FP64 operations per PE and block against K single steps: blocks must save 5 %
      const int64_t S = p.S[0], taps = 2 * p.h + 1;
      int64_t zone = 0;
      for (int j = 0; j + 1 < K; ++j) zone += 2 * zr[j];
      const int64_t block = zone * taps + (S - 8 * fe) * (2 * p.h * K + 1) + 8 * fe * taps;
      if (20 * block > 19 * K * S * taps) continue;
    }
    return K;
  }
  return 1;
}

void fuse_setup(StepParams *p, int k) {
  p->fuse_k = k > 1 ? k : 0;
  p->fe = 0;
  std::memset(p->zr, 0, sizeof(p->zr));
  std::memset(p->ck, 0, sizeof(p->ck));
  if (k <= 1) return;
  const int h = p->h;
  fuse_radii(h, k, &p->fe, p->zr);
  if (!p->use_pe[0]) p->fe = 0;
  // K-fold composition of the merged taps (s0 at the centre), in a fixed order
  double s[2 * AT_MAX_H + 1], c[2 * AT_MAX_H * AT_MAX_FUSE + 1] = {1.0}, t[2 * AT_MAX_H * AT_MAX_FUSE + 1];
  for (int j = -h; j <= h; ++j) s[j + h] = j == 0 ? p->s0 : p->s[0][j + h];
  int w = 0;  // c holds taps -w .. w at c[0 .. 2w]
  for (int step = 0; step < k; ++step) {
    const int w2 = w + h;
    for (int i = 0; i <= 2 * w2; ++i) t[i] = 0.0;
    for (int i = 0; i <= 2 * w; ++i)
      for (int j = 0; j <= 2 * h; ++j) t[i + j] += c[i] * s[j];
    w = w2;
    for (int i = 0; i <= 2 * w; ++i) c[i] = t[i];
  }
  for (int i = 0; i <= 2 * w; ++i) p->ck[i] = c[i];
}

cudaError_t launch_sync_rhs(const StepParams &p, const double *u, double *out, cudaStream_t st) {
  StepParams q = p;
  q.use_pe[0] = q.use_pe[1] = q.use_pe[2] = 0;  // no PE boundary: central differences at every point
  const bool grouped = grouped_shape(q, u) && (reinterpret_cast<uintptr_t>(out) % 16) == 0;
  const int64_t work = grouped ? q.ntot / 4 : q.ntot;
  const int64_t b = (work + 255) / 256, cap = (int64_t)sm_count() * 8;
  const int blocks = (int)(b < cap ? b : cap);
  const int g = grouped ? 1 : 0;
  if (q.dim == 1) {
    if (q.h == 1) sync_rhs_kernel<1, 1><<<blocks, 256, 0, st>>>(q, u, out, g);
    else if (q.h == 2) sync_rhs_kernel<1, 2><<<blocks, 256, 0, st>>>(q, u, out, g);
    else sync_rhs_kernel<1, 3><<<blocks, 256, 0, st>>>(q, u, out, g);
  } else {
    if (q.h == 1) sync_rhs_kernel<3, 1><<<blocks, 256, 0, st>>>(q, u, out, g);
    else if (q.h == 2) sync_rhs_kernel<3, 2><<<blocks, 256, 0, st>>>(q, u, out, g);
    else sync_rhs_kernel<3, 3><<<blocks, 256, 0, st>>>(q, u, out, g);
  }
  return cudaGetLastError();
}
