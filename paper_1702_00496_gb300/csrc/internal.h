// internal.h -- declarations shared by the translation units of libatfd (not part of the C ABI).
#pragma once
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/at.h"

#define AT_MAX_L 8
#define AT_MAX_T 4
#define AT_MAX_H 3
#define AT_MAX_MODES 16
#define AT_MAX_ETAPS 8
#define AT_MAX_KROT 64
#define AT_STAT_FIELDS 9
#define AT_STAT_BLOCKS 1024
#define AT_MAX_FUSE 4

void at_internal_set_error(const char *msg);

// Everything one forward step needs, passed to the kernel by value.
struct StepParams {
  double *ring;           // R slots of ntot doubles; level m in slot m mod R
  uint8_t *log;           // raw delays, step-major [log_steps][nb], or nullptr
  uint8_t *keff;          // effective delays, two buffers of nb: step n uses keff + (n & 1) * nb
  int64_t log_steps;      // rows of the log
  const int32_t *order;   // 3D: group visiting order (interior groups first, then edge groups), or nullptr
  int32_t *status;        // unused (null); kept so the fields after it keep the offsets the step kernels were
                          // tuned with
  double *frhs;           // Adams-Bashforth: ts-1 slots of ntot holding dt f^{n-m}, m = 1..ts-1, in slot
                          // (n-m) mod (ts-1); nullptr for forward Euler
  const int64_t *ab_first;  // device: first step whose right-hand side is stored (-(ts-1) after an analytic
                            // pre-history, 0 after a caller's field); steps before ts-1 stored levels use
                            // the lower-order weights
  int64_t ntot;           // points
  int64_t nb;             // PE sides, 2 * dim * prod(pe)
  int32_t n[3];           // points per axis
  int32_t S[3];           // PE width per axis
  int32_t pe[3];          // PEs per axis
  int32_t use_pe[3];      // axis has PE boundaries (pe > 1)
  int32_t dim, h, T, R, L, scheme;
  int32_t ts;             // time levels of the integrator: 1 forward Euler, 2 AB2, 3 AB3
  int32_t use_thr;        // thresholds given (else uniform bins)
  uint64_t seed;
  uint64_t thr[AT_MAX_L]; // L-1 bin edges on the 32-bit word
  int32_t threads;        // launch shape of the per-step kernel: threads per block
  int32_t blocks_per_sm;  // and a cap on blocks per SM for its grid-stride loop
  double zero;            // +0.0, kept opaque so the compiler issues an FMA rather than a multiply
  double s0;              // merged centre coefficient: 1 + dt sum_a (-c_a cd1_0/dx_a + alpha cd2_0/dx_a^2)
                          // (without the 1 for ts > 1, where the chain forms dt f^n)
  double beta[3][3];      // Adams-Bashforth weights beta[l-1][m] of dt f^{n-m} with l stored levels
  double s[3][2 * AT_MAX_H + 1];  // merged off-centre coefficients per axis (index j+h)
  double q0;                      // d s0 / d alpha = dt sum_a cd2_0 / dx_a^2
  double q[3][2 * AT_MAX_H + 1];  // d s_{a,j} / d alpha = dt cd2_j / dx_a^2
  double w[AT_MAX_L][AT_MAX_T];   // halo extrapolation weights w[k][m] of level n-k-m
  double sc[3];                   // per-axis centre coefficient s_{a,0} (s0 = 1 + sc[0] + sc[1] + sc[2])
  // Rows expanded in space (AT_AT_SPACE2 / AT_AT_SPACE1): merged taps dt (-c_a D1 + alpha D2) of the PE-edge
  // point of axis a, side s (0: buffer points on the left), at offset ej, read at level n (ebuf 0) or n-k
  // (ebuf 1); used when that side's delay is k > 0.
  int32_t ecount[3][2];
  int8_t ej[3][2][AT_MAX_ETAPS];
  int8_t ebuf[3][2][AT_MAX_ETAPS];
  double ec[3][2][AT_MAX_ETAPS];
  // Burgers' equation.  New fields go at the end: the offsets of the fields above are those the linear step
  // kernels were tuned with (inserting these earlier slowed the 1D order-4 step by 3 %, 165 against 160 us).
  int32_t burgers;                // 1: viscous Burgers' equation, f = -u D1 u + alpha D2 u (1D)
  double b1[2 * AT_MAX_H + 1];    // Burgers: dt cd1_j / dx (index j+h; the first derivative's taps)
  double b2[2 * AT_MAX_H + 1];    // Burgers: dt alpha cd2_j / dx^2
  // For the adjoint's alpha term: the per-axis centre dt cd2_0 / dx_a^2 (q0 is their sum) and the second-derivative
  // part dt c2 / dx_a^2 of each merged edge-row tap of the rows expanded in space.
  double qc[3];
  double eq[3][2][AT_MAX_ETAPS];
  // K-step blocks of the 1D forward-Euler step (central and time-expanded rows, groups of four), fuse_k = K > 1:
  // step j < K-1 of a block computes only the cells within zr[j] of every PE boundary, step K-1 the edge groups
  // (fe per PE end) from U^{n+K-1} and every other group from U^n with ck, the K-fold composition of the merged
  // interior taps (index j + h K).
  int32_t fuse_k, fe;
  int32_t zr[AT_MAX_FUSE];
  double ck[2 * AT_MAX_H * AT_MAX_FUSE + 1];
  // Host: the first step whose Adams-Bashforth combination has all ts levels stored (0 after the analytic
  // pre-history, ts-1 from a caller's field); from it on the weights are beta[ts-1] at every step, and AB2 steps
  // take the combination's steady form.
  int64_t ab_steady;
};

// The modes of one axis at one time t, prepared on the host for the recurrences over k: sorted by wavenumber,
// with A exp(-alpha kappa^2 t) and the phase phi - kappa c t folded into ac = A cos(.), as = A sin(.).  rot = 1 when
// every wavenumber is an integer in 1..AT_MAX_KROT (else the sines are evaluated one by one).
struct ModeSet {
  int32_t rot, kmax;
  int32_t kr[AT_MAX_MODES];
  double ac[AT_MAX_MODES], as[AT_MAX_MODES];
};
void fill_modes(ModeSet *ms, const double *amp, const double *phase, const double *kappa, int nmodes, double alpha,
                double c, double t);

// Initial-condition / analytic-solution parameters.
struct WaveParams {
  int32_t dim, nmodes;
  int32_t n[3];
  double dx[3];
  double c[3];
  double alpha;
  double amp[3][AT_MAX_MODES];
  double phase[3][AT_MAX_MODES];
  double kappa[3][AT_MAX_MODES];
  ModeSet ms[3];  // per axis, filled by the launchers for the time of the launch (fill_modes)
  double xpi[3];  // 2 / n: grid point i sits at x = pi (i xpi)
};

// Validate cfg and fill the step parameters (merged taps, extrapolation weights, delay process) for a problem
// whose ring starts at ring_dev; log_dev (log_steps rows) may be null.  The caller sets keff.  Host only.
int at_prepare_params(const at_config_t *cfg, double *ring_dev, uint8_t *log_dev, int64_t log_steps, StepParams *out);

// Launchers (return cudaGetLastError()).
// One forward step n = n_off + (*n_base if n_base else 0): reading the base from device memory lets a
// captured graph of consecutive steps be replayed at any step.
cudaError_t launch_forward_step(const StepParams &p, int64_t n_off, const int64_t *n_base, cudaStream_t st);
// The fuse_k steps n .. n+fuse_k-1 of a block (n = n_off + *n_base): zone launches, then the block launch.
cudaError_t launch_forward_block(const StepParams &p, int64_t n_off, const int64_t *n_base, cudaStream_t st);
// Largest block length K <= kmax (1: none) that the problem admits, and the block parameters for K (host).
int fuse_max_k(const StepParams &p, const void *ring, int kmax);
void fuse_setup(StepParams *p, int k);
// *n_base = v (set) or *n_base += v.
cudaError_t launch_step_counter(int64_t *n_base, int64_t v, bool set, cudaStream_t st);
// Draw the delays of step n into keff + (n & 1) * nb (and log row n): the set-up before a first step.
cudaError_t launch_draw_delays(const StepParams &p, int64_t n, cudaStream_t st);
// Adams-Bashforth pre-history: dt f of the field u with synchronous stencils into out (ntot doubles).
cudaError_t launch_sync_rhs(const StepParams &p, const double *u, double *out, cudaStream_t st);
cudaError_t launch_wave_field(const WaveParams &w, double t, double *tables, double *out, cudaStream_t st);
cudaError_t launch_error_stats(const WaveParams &w, const StepParams &p, const double *u, double t,
                               double *tables, double *partials, double *result, cudaStream_t st);
// The same statistics of E = U - V for a reference field V `refine` times finer on every axis.
cudaError_t launch_error_stats_ref(const WaveParams &w, const StepParams &p, const double *u, const double *ref,
                                   int refine, double *partials, double *result, cudaStream_t st);

// The solver handle behind at_handle_t (shared by api.cu and adjoint.cu).
struct at_handle {
  at_config_t cfg;
  std::vector<uint64_t> thr;
  StepParams sp;
  WaveParams wp;
  int64_t log_steps = 0;
  int64_t step = 0;
  cudaStream_t stream = nullptr;
  // scratch owned by the handle: step counter, reduction partials and result, 3D axis tables
  void *scratch = nullptr;
  double *d_partials = nullptr;
  double *d_result = nullptr;
  double *d_tables = nullptr;
  int64_t *d_step = nullptr;  // step base read by the captured graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // adjoint state: the forward pass with checkpoints records its schedule here
  int64_t adj_nsteps = -1;       // steps of the checkpointed forward pass (-1: none)
  int64_t adj_every = 0;         // checkpoint interval
  double *adj_work = nullptr;    // caller's workspace
  int64_t adj_work_len = 0;
  bool ab_analytic = false;      // Adams-Bashforth run started from Eq. "IC" with the analytic pre-history
  bool adj_resident = false;     // the forward pass kept every level in the workspace (one segment)
  int64_t n_interior = 0;        // 3D grouped shapes: interior groups at the head of sp.order
};

// Steps per captured graph: long runs replay one graph of kGraphSteps kernel nodes plus a counter update.
static const int64_t kGraphSteps = 50;
