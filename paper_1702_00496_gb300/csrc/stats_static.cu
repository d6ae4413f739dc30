// stats_static.cu -- the error-statistics reduction without any allocation.
//
// at_error_stats needs a solver handle, and creating a handle allocates device scratch.  Some callers cannot
// allocate device memory at all: code running under a memory pool that forbids new cudaMalloc calls after start
// up, an embedding that hands this library only the buffers it owns, or a process sitting close to its memory
// limit.  at_error_stats_noalloc computes the same statistics of a field the caller already has, using a block of
// scratch that lives in this library's own device memory image: the file-scope array below.  Every GPU that loads
// the library holds that array (about 270 KB) until the process exits.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda.h>  // CUcontext and the driver's result type only: the two driver calls are looked up at run time

#include "../../include/at.h"
#include "internal.h"

namespace {

// Scratch of the reduction: per-block partials, the final sums, and (3D) the per-axis tables of the analytic
// solution.  Every call overwrites what it uses before reading it, so nothing has to start at zero.
constexpr int kPartials = AT_STAT_BLOCKS * AT_STAT_FIELDS;
constexpr int kResult = 16;
constexpr int kMaxTables = 3 * 8192;
constexpr int kScratchDoubles = kPartials + kResult + kMaxTables;

__device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// The array's device address, looked up with cudaGetSymbolAddress once per CUDA context and kept per device
// together with the id of the context it belongs to.  A device reset (cudaDeviceReset by the caller or by
// another library) destroys the context and the module image with it; the next call then sees a new context id
// and looks the address up again instead of using the stale one.  The mutex makes the look-up safe when several
// host threads call at once.
constexpr int kMaxDevices = 64;
struct ScratchAddr {
  unsigned long long ctx_id;
  double *addr;
};
ScratchAddr g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
std::once_flag g_driver_once;

// Id of the context current on this thread (0 when none is, or the driver does not offer the calls).
unsigned long long current_context_id() {
  std::call_once(g_driver_once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f);
  });
  if (!g_ctx_get_current || !g_ctx_get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return 0;
  if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
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

const double kTwoPi = 6.283185307179586476925286766559005768;

}  // namespace

extern "C" int at_error_stats_noalloc(const at_config_t *cfg, const double *u_dev, int64_t step, void *stream,
                                      at_stats_t *out) {
  int32_t R;
  int rc = at_ring_slots(cfg, &R);  // validates cfg; host only, allocates nothing
  if (rc) return rc;
  if (!u_dev || !out || step < 0) return fail(AT_ERR_ARG, "at_error_stats_noalloc: bad argument");
  if (cfg->burgers) return fail(AT_ERR_ARG, "at_error_stats_noalloc: Burgers' equation has no analytic solution here");
  if (cfg->dim == 3 && cfg->n[0] + cfg->n[1] + cfg->n[2] > kMaxTables)
    return fail(AT_ERR_ARG, "at_error_stats_noalloc: n[0]+n[1]+n[2] exceeds 24576 (the static scratch limit)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "at_error_stats_noalloc: device");
  if (dev < 0 || dev >= kMaxDevices) return fail(AT_ERR_ARG, "at_error_stats_noalloc: device index beyond 63");
  // once per device and context, with that device current: the device address of the static scratch.  The
  // runtime makes the device's primary context current on the first call that needs it; before that, no
  // context id is known, and the address is looked up (which makes the context current) and cached after.
  double *partials = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    unsigned long long ctx = current_context_id();
    ScratchAddr &slot = g_scratch_addr[dev];
    if (ctx != 0 && slot.addr != nullptr && slot.ctx_id == ctx) {
      partials = slot.addr;
    } else {
      void *ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "at_error_stats_noalloc: cudaGetSymbolAddress");
      partials = static_cast<double *>(ptr);
      if (ctx == 0) ctx = current_context_id();
      slot.ctx_id = ctx;
      slot.addr = ctx != 0 ? partials : nullptr;  // without a context id nothing is cached
    }
  }
  double *result = partials + kPartials;
  double *tables = result + kResult;

  StepParams p;
  std::memset(&p, 0, sizeof(p));
  p.ntot = cfg->n[0] * cfg->n[1] * cfg->n[2];
  p.dim = cfg->dim;
  p.h = cfg->order / 2;
  WaveParams w;
  std::memset(&w, 0, sizeof(w));
  w.dim = cfg->dim;
  w.nmodes = cfg->nmodes;
  w.alpha = cfg->alpha;
  for (int a = 0; a < 3; ++a) {
    p.n[a] = (int32_t)cfg->n[a];
    p.pe[a] = cfg->pe[a];
    p.S[a] = (int32_t)(cfg->n[a] / cfg->pe[a]);
    p.use_pe[a] = (a < cfg->dim && cfg->pe[a] > 1) ? 1 : 0;
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
  cudaStream_t st = (cudaStream_t)stream;
  e = launch_error_stats(w, p, u_dev, (double)step * cfg->dt, tables, partials, result, st);
  if (e != cudaSuccess) return cuda_fail(e, "at_error_stats_noalloc: launch");
  double r[AT_STAT_FIELDS];
  if ((e = cudaMemcpyAsync(r, result, sizeof(r), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_fail(e, "at_error_stats_noalloc: copy");
  const double N = (double)p.ntot;
  out->rms = std::sqrt(r[0] / N);
  out->max_abs = r[1];
  out->mean_abs = r[2] / N;
  out->mean = r[3] / N;
  out->rms_I = r[7] > 0 ? std::sqrt(r[4] / r[7]) : 0.0;
  out->rms_B = r[8] > 0 ? std::sqrt(r[5] / r[8]) : 0.0;
  out->ua_rms = std::sqrt(r[6] / N);
  out->n_I = (int64_t)r[7];
  out->n_B = (int64_t)r[8];
  out->step = step;
  if (!std::isfinite(out->rms) || !std::isfinite(out->max_abs))
    return fail(AT_ERR_NONFINITE, "at_error_stats_noalloc: non-finite error");
  return AT_OK;
}
