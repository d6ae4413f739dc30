/*
 * at.h -- C ABI of the GB300 (sm_103a) implementation of the asynchrony-tolerant (AT)
 * finite-difference method of Aditya & Donzis (arXiv:1702.00496).
 *
 * The hot path is the explicit forward-Euler step (Sec. 4.1, Eq. "time_disc" with one level; Adams-Bashforth
 * with two or three levels on request) of
 *     u_t + c . grad u = alpha lap u
 * on a periodic box [0, 2 pi)^dim (Sec. 5.1), split into emulated processing elements (PEs,
 * Sec. 2).  Interior points use central differences (Eq. "general_deriv_cds"); points within the
 * stencil half-width of a PE boundary use AT stencils (Tables "atschemes-left/right"), which read
 * the neighbouring PE's values at delayed time levels n-k, n-k-1, ... with k drawn per PE side per
 * step (Sec. 5.1, "simulate delays").
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int status: AT_OK (0) or a negative AT_ERR_* code.  Nothing throws,
 *     aborts or traps; at_last_error() gives a one-line message for the calling thread.
 *   - Pointers named *_dev are CUDA device pointers, owned by the caller (e.g. torch tensors); the
 *     library borrows them for the lifetime of the handle.  Pointers named *_host are host memory.
 *   - Fields are FP64, row-major with x fastest: index (z*ny + y)*nx + x.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Work is enqueued
 *     asynchronously unless the function says it blocks.
 *   - A handle may be used by one host thread at a time.
 */
#ifndef ATFD_AT_H
#define ATFD_AT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AT_OK 0
#define AT_ERR_ARG (-1)          /* invalid argument, detected on the host before any launch */
#define AT_ERR_SINGULAR (-2)     /* Sec. 3.2: rank(A) = rank(A|b) < N_A -- infinitely many schemes */
#define AT_ERR_INCONSISTENT (-3) /* Sec. 3.2: rank(A) != rank(A|b) -- the stencil gives no scheme */
#define AT_ERR_CUDA (-4)         /* a CUDA runtime call failed */
#define AT_ERR_TIMEOUT (-5)      /* reserved: no kernel of this library waits on a flag or a peer, so none returns it */
#define AT_ERR_NONFINITE (-6)    /* a statistic came out NaN or Inf */
#define AT_ERR_BOUNDS (-7)       /* reserved: every index a kernel forms is in range by construction (sizes, PE
                                  * widths, delays and the log length are checked on the host before any launch),
                                  * so no kernel reports one */
#define AT_ERR_STATE (-8)        /* call out of order, e.g. more steps than the delay log holds */

/* Spatial scheme at PE boundaries. */
#define AT_SYNC 0      /* every delay is 0: standard central differences everywhere (Eq. "general_deriv") */
#define AT_ASYNC_STD 1 /* central differences read at the delayed level n-k (Eq. "general_deriv_async") */
#define AT_AT 2        /* asynchrony-tolerant, time-expanded stencils ((1,2,2)b/(2,2,2)b, (1,4,2)/(2,4,2), (2,6,2)) */
#define AT_AT_SPACE2 3 /* AT stencils expanded in space, (1,2,2)a/(2,2,2)a (Case 3): order 2, forward Euler; the
                        * PE-edge point of a side with delay k > 0 uses the row, k = 0 the central difference */
#define AT_AT_SPACE1 4 /* the first-order row expanded in space, (2,1,2) (Case 2): order 2, forward Euler, diffusion
                        * only (c = 0); edge rows for k > 0 as for AT_AT_SPACE2 */

/* ------------------------------------------------------------------ scheme coefficients */
typedef struct {
  int32_t deriv;  /* d: 1 or 2 */
  int32_t order;  /* a: 2, 4 or 6 (spatial order of accuracy) */
  int32_t L;      /* delays take values 0..L-1, L <= 8 */
  int32_t h;      /* half-width of the central stencil, a/2 */
  int32_t T;      /* successive delayed levels read at a buffer point, 1 + #{q >= 1 : 2q < d + a} */
  double cd[9];   /* per-point central weights for offsets j=-h..h at cd[j+h], in units of 1/dx^d */
  int64_t cd_num[9], cd_den;   /* the same weights as exact fractions cd_num[j+h] / cd_den */
  double phi[5];  /* stage-1 weights phi_0..phi_h on (u_{i+j} + (-1)^d u_{i-j}), Eq. "general_deriv_cds" */
  double w[8][4]; /* stage-2 weights w[k][m] of the copy read at level n-k-m, m < T (Example 3) */
  int64_t w_num[8][4], w_den[8]; /* w[k][m] = w_num[k][m] / w_den[k] exactly */
} at_coeffs_t;

/* Derive the AT scheme of derivative `deriv` and order `order` for delays 0..L-1 by the two-stage
 * procedure of Sec. 3.3 (Example 3): stage 1 solves the symmetric-pair system of Eq. "general_deriv_cds"
 * for the central weights, stage 2 solves, for each k, the time-level system that cancels the
 * asynchronous Taylor terms u^(p,q), q >= 1, p + 2q < d + a (Eq. "cond", dt ~ dx^2).  Both systems are
 * solved in exact rational arithmetic with the rank tests of Sec. 3.2, and the expanded coefficients
 * are re-checked against every condition of Eq. "cond".  Host only; no CUDA call.
 * Errors: AT_ERR_ARG (deriv not 1/2, order not 2/4/6, L outside 1..8, out NULL), AT_ERR_SINGULAR,
 * AT_ERR_INCONSISTENT. */
int at_coeffs(int32_t deriv, int32_t order, int32_t L, at_coeffs_t *out);

/* Expanded taps c~_{j,l} (Eq. "general_deriv_at2") of derivative `deriv` at a point `pos` cells in
 * from a PE edge (pos = 0 is the edge point) on side `side` (0: buffer points on the left, 1: on the
 * right), for scheme AT_SYNC / AT_ASYNC_STD / AT_AT / AT_AT_SPACE2 / AT_AT_SPACE1 and effective delay k.  The rows
 * expanded in space are derived from their shapes ({i+1, i; i-1, i-2} for (1,2,2)a and (2,1,2), {i+2, i+1, i; i-1,
 * i-2, i-3} for (2,2,2)a, buffer points at level n-k, mirrored for side 1) by the single system of Sec. 3.1-3.2.
 * Coefficients are in units of 1/dx^d, taps with equal (j, l) merged.  Writes at most `cap` taps (j_out, l_out,
 * c_out) and stores their number in *ntaps.  Host only.  Errors: AT_ERR_ARG (also: AT_AT_SPACE1 with deriv 1 at
 * an edge point with k > 0, the space schemes with order != 2). */
int at_stencil_taps(int32_t deriv, int32_t order, int32_t scheme, int32_t k, int32_t pos, int32_t side,
                    int32_t cap, int32_t *j_out, int32_t *l_out, double *c_out, int32_t *ntaps);

/* The general single-system derivation of Sec. 3.1-3.2: impose Eq. "cond" (rows p + r q < d + a) on the
 * stencil {(j_i, l_i)}, i < npts (point i+j read at level n-l), and solve A c = b exactly.
 * On AT_OK, num_out[i]/den_out[i] and c_out[i] hold the unique coefficients (units 1/dx^d, dt = dx^r
 * taken as 1 in the row scaling).  *rank_out receives rank(A) in every case.
 * Errors: AT_ERR_ARG (npts outside 1..32, bad d/a/r), AT_ERR_SINGULAR (consistent, rank deficient),
 * AT_ERR_INCONSISTENT (rank(A) != rank(A|b)).  Host only. */
int at_solve_stencil(int32_t deriv, int32_t order, int32_t r, int32_t npts, const int32_t *j, const int32_t *l,
                     int64_t *num_out, int64_t *den_out, double *c_out, int32_t *rank_out);

/* ------------------------------------------------------------------ delay process */
/* Raw delay of PE side `side` at step `step` (Sec. 5.1): the first word x0 of Philox4x32-10 with
 * counter (step, side, 0, 0) and key (seed_lo, seed_hi) is binned -- uniformly, k = floor(x0 L / 2^32),
 * when thresholds_host is NULL, else k = #{m < L-1 : thresholds_host[m] <= x0}.  Host-side copy of the
 * generator the kernels run, for replay and tests.  Returns k >= 0, or AT_ERR_ARG. */
int at_delay(uint64_t seed, int64_t step, int64_t side, int32_t L, const uint64_t *thresholds_host);

/* ------------------------------------------------------------------ problem and handle */
typedef struct {
  int32_t dim;     /* 1 or 3 */
  int32_t order;   /* 2, 4 or 6 */
  int32_t L;       /* delays 0..L-1, 1 <= L <= 8 */
  int32_t scheme;  /* AT_SYNC, AT_ASYNC_STD, AT_AT, AT_AT_SPACE2 or AT_AT_SPACE1 */
  int64_t n[3];    /* points per axis (axes beyond dim hold 1) */
  int32_t pe[3];   /* PEs per axis; n[a] % pe[a] == 0 and n[a]/pe[a] >= order.  pe[a] == 1: no boundary */
  int32_t nmodes;  /* initial-condition modes per axis, 1..16 */
  double c[3];     /* advection speed per axis */
  double alpha;    /* diffusivity */
  double dt;       /* time step */
  uint64_t seed;   /* delay-process key */
  const uint64_t *thresholds; /* host, L-1 ascending values in [0, 2^32], or NULL for uniform delays */
  const double *amp;          /* host [dim][nmodes]: A in Eq. "IC" */
  const double *phase;        /* host [dim][nmodes]: phi in Eq. "IC" */
  const int32_t *kappa;       /* host [dim][nmodes]: wavenumbers in Eq. "IC" */
  int32_t tsteps;  /* time integrator (Sec. 4.1, Eq. "time_disc"): 0 or 1 forward Euler, 2 Adams-Bashforth with two
                    * levels (Eq. "time_ab2"), 3 with three levels (weights 23/12, -16/12, 5/12).  A multistep run
                    * from Eq. "IC" takes the right-hand sides of the tsteps-1 levels before t = 0 from the analytic
                    * solution (central differences), so every step has full order; from a caller's field
                    * (at_reset with u0_dev) it starts with forward Euler and raises the order step by step. */
  int32_t burgers; /* 0: u_t + c . grad u = alpha lap u; 1: the viscous Burgers' equation u_t + u u_x = alpha u_xx
                    * (Sec. 5.1, Eq. "general" with beta_1 = u, beta_2 = alpha; Case 6): 1D, c = 0, schemes AT_SYNC,
                    * AT_ASYNC_STD or AT_AT; D1 and D2 use the same AT stencils, u_i is the point's current value.
                    * A multistep Burgers run starts with forward Euler (there is no analytic pre-history). */
} at_config_t;

typedef struct at_handle at_handle_t;

/* Ring-buffer slots R = L + T + (tsteps > 1 ? tsteps - 1 : 0): L + T solution levels (T from at_coeffs for this
 * order and scheme; 1 for SYNC/ASYNC_STD), then, for Adams-Bashforth, the stored right-hand sides dt f^{n-m}
 * (m = 1..tsteps-1).  at_num_sides: the number of PE sides 2*dim*prod(pe).  Host only.  Errors: AT_ERR_ARG. */
int at_ring_slots(const at_config_t *cfg, int32_t *R);
int at_num_sides(const at_config_t *cfg, int64_t *sides);

/* Create a solver on caller-owned device memory and write U^0 (Eq. "IC"; the 3D field is the product
 * of per-axis sums) into ring slot 0.
 *   ring_dev : R * n0*n1*n2 doubles (R from at_ring_slots), 16-byte aligned for the vectorised kernels (any
 *              other alignment runs the per-point kernel: the same results, slower); level m
 *              lives in slot m mod (L + T), the right-hand sides of Adams-Bashforth in the slots after those.
 *   log_dev  : log_steps * sides bytes, may be NULL when log_steps == 0; receives the raw delay of
 *              every PE side at every step (step-major), so each run can be replayed and audited.
 * The handle copies cfg and its host arrays and allocates a small scratch block for reductions.
 * Errors: AT_ERR_ARG, AT_ERR_CUDA. */
int at_init(const at_config_t *cfg, double *ring_dev, int64_t ring_len, uint8_t *log_dev, int64_t log_steps,
            void *stream, at_handle_t **out);

/* Advance nsteps steps (the hot path; forward Euler or Adams-Bashforth per cfg->tsteps).  Each step draws the delays of every PE side,
 * extrapolates the halo each side reads from the delayed ring slots, and applies the fused stencil.
 * 1D forward-Euler problems with the central or time-expanded rows advance in blocks of K steps where the shape
 * allows it (at_set_fusion): inside a PE, away from its boundaries, K steps of the constant interior stencil are
 * one stencil of half-width h K (the K-fold composition of its taps; exact in exact arithmetic, the rounding of
 * each cell differs), and the cells near PE boundaries, which read delayed halo values, are stepped one step at a
 * time; the delays, the delay log and the levels a later step reads at delayed levels are those of single steps.
 * Blocks start at the first step of each call (and of each captured graph inside it, 48 steps for K = 4), so the
 * same steps split into other calls give results equal up to rounding, not bit for bit.
 * Adams-Bashforth runs from a caller's field take their first ts-1 steps (fewer stored levels, other weights) as
 * single launches; every later step -- every step after the analytic pre-history -- has all ts levels (with ts = 2
 * its weights are then read as kernel parameters: the same operations, the same bits).
 * Enqueued on the handle's stream; returns without waiting.  Errors: AT_ERR_ARG, AT_ERR_STATE (the
 * delay log would overflow), AT_ERR_CUDA. */
int at_step(at_handle_t *hd, int64_t nsteps);

/* Block length of at_step for the following calls: the largest K <= k (1..4) the problem admits -- 1D, forward
 * Euler, AT_SYNC / AT_ASYNC_STD / AT_AT, not Burgers, n0 and the PE width multiples of 4, ring 16-byte aligned,
 * more ring slots than K, and PEs wide enough that the zones stepped one step at a time (under 10 h + 16 cells
 * around each boundary for K = 4) do not meet and that a block saves at least 5 % of the FP64 operations of K
 * single steps (PEs of at least 144 cells for order 4 and K = 4, 72 for order 2) -- written to *k_used (1: single
 * steps).  at_init picks the largest
 * admissible K <= 4.  k = 1 restores single steps.  Waits for the stream and drops the captured step graph.
 * Errors: AT_ERR_ARG (k outside 1..4), AT_ERR_CUDA. */
int at_set_fusion(at_handle_t *hd, int32_t k, int32_t *k_used);

/* Restart at step 0: write U^0 into ring slot 0 -- Eq. "IC" when u0_dev is NULL, else a copy of the
 * caller's field u0_dev (n0*n1*n2 doubles, device) -- and rewind the step counter.  The delay process
 * replays from step 0.  Enqueued on the handle's stream.  Errors: AT_ERR_ARG, AT_ERR_CUDA. */
int at_reset(at_handle_t *hd, const double *u0_dev);

/* Launch shape of the per-step kernel for the following at_step calls: threads per block (128, 256 or 512)
 * and a cap of blocks_per_sm (1..64) blocks per SM on its grid-stride loop.  Defaults 256 and 32.  Waits
 * for the stream and drops the captured step graph.  Used by the autotuner.  Errors: AT_ERR_ARG. */
int at_set_launch(at_handle_t *hd, int32_t threads, int32_t blocks_per_sm);

/* Wait for the handle's stream.  Returns AT_OK, or AT_ERR_CUDA with the runtime's message when the stream reports
 * an error (a failed launch or copy).  Blocks. */
int at_sync(at_handle_t *hd);

/* Current step n and a device pointer to U^n inside the ring (valid until the next at_step). */
int at_state(at_handle_t *hd, int64_t *step, double **field_dev);

/* Sec. 4 / Sec. 5.1 error measures of E = U^n - u_a(x, n dt), where u_a is Eq. "ana_sol" read as
 * sum A exp(-alpha kappa^2 t) sin(kappa (x - c t) + phi) (3D: product over axes).  rms is over all
 * points, rms_I / rms_B over the interior set I_I and the PE-boundary set I_B (points within h of a
 * boundary of a split axis).  Deterministic two-pass reduction.  Blocks.  Errors: AT_ERR_CUDA,
 * AT_ERR_NONFINITE. */
typedef struct {
  double rms, max_abs, mean_abs, mean, rms_I, rms_B, ua_rms;
  int64_t n_I, n_B, step;
} at_stats_t;
int at_error_stats(at_handle_t *hd, at_stats_t *out);

/* The statistics of E = U^n - V for a caller's reference field V (device, 16-byte aligned) on a grid `refine`
 * (>= 1) times finer on every axis of the problem -- n0*refine x n1*refine x n2*refine doubles for dim 3,
 * n0*refine for dim 1 -- sampled at the coarse points (V at (refine x, refine y, refine z)); ua_rms is the RMS of
 * the sampled reference.  The paper measures its Burgers runs (no analytic solution) this way, against a finer
 * run.  at_error_stats rejects Burgers problems (AT_ERR_ARG); this entry point takes any problem.  Blocks.
 * Errors: AT_ERR_ARG, AT_ERR_CUDA, AT_ERR_NONFINITE. */
int at_error_stats_ref(at_handle_t *hd, const double *ref_dev, int32_t refine, at_stats_t *out);

/* The statistics of at_error_stats for a field the caller holds (u_dev: device, n0*n1*n2 doubles of the problem
 * cfg at step `step`, t = step * dt), computed without allocating anything.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory -- a process under a memory pool that refuses
 * new allocations after start-up, an embedding that gives the library only buffers it owns, or a job close to
 * its memory limit -- and so cannot create a handle (at_init allocates scratch).
 * Scratch: one static device array of this library (33,808 doubles, about 270 KB), held by every GPU that loads
 * the library until the process exits.  3D problems need n[0] + n[1] + n[2] <= 24576; larger ones are rejected
 * with AT_ERR_ARG.  Each call overwrites the scratch it reads, so nothing must be cleared between calls, but every
 * call shares the one array: calls that overlap on the GPU (different streams or host threads) race.  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress) with that device current and keeps
 * it for the device's current CUDA context; make that first call before any stream capture.  A device reset ends
 * that context: the next call looks the address up again (so it, too, belongs before any capture).  No cudaMalloc, cudaFree or other allocating call is made.  Blocks
 * on `stream` (a cudaStream_t, NULL = default stream).  Errors: AT_ERR_ARG, AT_ERR_CUDA, AT_ERR_NONFINITE. */
int at_error_stats_noalloc(const at_config_t *cfg, const double *u_dev, int64_t step, void *stream, at_stats_t *out);

/* Release the handle's scratch.  The caller's ring and log are untouched. */
int at_destroy(at_handle_t *hd);

/* ------------------------------------------------------------------ adjoint */
/* Gradient of a misfit J(U^nsteps) with respect to the initial field U^0 and the diffusivity alpha, through the
 * same delays as the forward run.  The forward step is linear in the stored levels; its transpose sends
 * lambda^{n+1} back through the merged taps to lambda^n and, for buffer points, through the extrapolation
 * weights w_m(k) of the replayed delay k to lambda^{n-k-m}.  dJ/dalpha = sum_n <lambda^{n+1}, dt D2_AT U^n>.
 * The paper has no adjoint; this is the exact discrete adjoint of the forward step of Sec. 4.1 / Tables
 * "atschemes-left/right" for orders 2, 4 and 6, every scheme, the linear equation
 * and Burgers' equation (whose transpose is state-dependent: the first-derivative taps carry -U_i^n and U_i^n
 * itself receives -D1 U, so the backward sweep always recomputes the forward levels), with forward Euler or
 * Adams-Bashforth, and for the rows expanded in space (AT_AT_SPACE2 / AT_AT_SPACE1: each edge row's taps send
 * lambda to level n or n-k).  An Adams-Bashforth run must start
 * from a caller's field (at_reset with u0_dev; the analytic pre-history of a run from Eq. "IC" depends on alpha):
 * otherwise AT_ERR_STATE.  Its step n sends lambda^{n+1} to lambda^n (identity) and the adjoint of dt f^n,
 * mu^n = sum_m beta_m lambda^{n+1+m} over the later steps that use f^n, back through the transposed taps.
 *
 * at_adjoint_workspace: doubles of device workspace for a run of nsteps with a checkpoint every ckpt_every
 *   steps (0: ceil(sqrt(nsteps))): the checkpoints, one segment of recomputed levels, the R-slot adjoint ring and
 *   small accumulators.  A checkpoint at step n0 holds U^{n0} in full and, of the R-2 older levels the next steps
 *   read, only the cells within the buffer reach of a PE face along a split axis (h cells; 3 for the rows expanded
 *   in space): the only cells a step reads at delayed levels (Eq. "general_deriv_async").  At 256^3 in 4^3 PEs,
 *   order 4, L = 3 that is 17.6 % of the cells, so a checkpoint takes 1.7 fields instead of 5; Adams-Bashforth
 *   checkpoints also hold the ts-1 stored right-hand sides in full.
 * at_adjoint_forward: from step 0 (after at_init or at_reset), run nsteps forward steps one at a time (as at_step
 *   does with at_set_fusion(hd, 1, ...)) and keep the checkpoints in work_dev (caller-owned, 16-byte aligned, untouched until at_adjoint_backward).  When
 *   one segment covers the run (ckpt_every >= nsteps; workspace about nsteps + R fields), the steps run inside the
 *   workspace, which then holds every level, and the backward sweep recomputes nothing.  Any later at_step or
 *   at_reset discards the recorded pass.  Errors: AT_ERR_ARG, AT_ERR_STATE (not at step 0, or nsteps beyond the
 *   delay log or the 32-bit step counter, checked before any step), AT_ERR_CUDA.
 * at_adjoint_backward: given lambda_dev = dJ/dU^nsteps (device, ntot doubles), write dJ/dU^0 to grad_u0_dev
 *   (device, ntot doubles) and dJ/dalpha to *grad_alpha_host.  Replays one checkpoint segment at a time:
 *   restores it, recomputes its levels with the forward kernel, runs its adjoint steps in reverse (one launch
 *   per step); with every level in the workspace it only runs the adjoint steps.  With grad_alpha_host NULL
 *   only dJ/dU^0 is formed; the linear transposed steps need no forward level then, so the sweep skips the
 *   restore and the recompute.  dJ/dalpha is summed per block in a fixed assignment: deterministic.  Blocks.
 *   Requires at_adjoint_forward to have been the last stepping call.  Errors: AT_ERR_ARG, AT_ERR_STATE,
 *   AT_ERR_CUDA, AT_ERR_NONFINITE. */
int at_adjoint_workspace(at_handle_t *hd, int64_t nsteps, int64_t ckpt_every, int64_t *work_len);
int at_adjoint_forward(at_handle_t *hd, int64_t nsteps, int64_t ckpt_every, double *work_dev, int64_t work_len);
int at_adjoint_backward(at_handle_t *hd, const double *lambda_dev, double *grad_u0_dev, double *grad_alpha_host);

/* ------------------------------------------------------------------ batched ensemble */
/* The error of an AT scheme is a statistical quantity (Sec. 4: ensemble average over delay realizations,
 * Eq. "aveE_split"; Sec. 5.1: averages over runs with random phases; Sec. 5.2, Figs. "at-ord2-procs" and
 * "at-kmom": error against P, N and the delay moments, and the asynchronous part E - E_s against a synchronous
 * but otherwise identical run).  An ensemble runs `count` independent 1D problems -- each with its own n[0] and
 * PE width (multiples of 4), order, time integrator, L, delay probabilities, seed, initial condition, dt and step
 * count -- inside one persistent kernel captured in a CUDA graph: CTAs take realizations from a work counter in
 * longest-first order (cost n[0] x steps), so uneven runs balance over the SMs.
 *
 * at_member_t describes how member r runs:
 *   nsteps : steps it runs (0..2^32-1); its statistics are taken at t = nsteps * dt.
 *   group  : label of its summary group (>= 0), or -1 for "its grid size n[0]"; the summary averages over the
 *            members that share a key (the label, or n[0]).
 *   twin   : index of another member with the same n[0] whose final field this member's final field is compared
 *            with (RMS and mean absolute value over the points of U - U_twin; e.g. its synchronous twin, so the
 *            asynchronous part of the error is measured on the same initial condition), or -1.
 *
 * at_ensemble_sizes: validates the members and runs and gives the doubles of ring and bytes of delay log they
 *   need (members stored one after another; member r's ring holds its own at_ring_slots slots, its log
 *   nsteps_r x sides_r bytes).
 * at_ensemble_create: members and runs are copied; ring_dev (ring_len doubles, 16-byte aligned) and the optional
 *   log_dev (log_len bytes, NULL for no log) are borrowed.  threads per CTA is 128, 256, 512 or 1024 (0: 1024);
 *   ctas_per_sm <= 0 takes the occupancy limit.  Every member starts from Eq. "IC" (with the analytic
 *   pre-history for Adams-Bashforth).  Errors: AT_ERR_ARG (non-1D member, n[0] or the PE width not a multiple
 *   of 4, bad nsteps, group or twin, sizes), AT_ERR_CUDA.
 * at_ensemble_run: one graph launch on the ensemble's stream (asynchronous).
 * at_ensemble_stats: blocks; per_member[r] (up to cap entries) receives member r's error statistics at its final
 *   step (the at_error_stats fields) and per_member_diff[2r], [2r+1] the RMS and the mean absolute value of
 *   U - U_twin (0 without a twin); groups[g] (g < *ngroups, ascending keys, up to gcap entries) the group's key,
 *   member count, the ensemble mean and unbiased variance of the members' RMS errors, the mean of their mean
 *   absolute errors and, over its members with a twin, mean and variance of both twin differences.
 *   Any output pointer but ngroups may be NULL.  Errors: AT_ERR_CUDA, AT_ERR_NONFINITE. */
typedef struct at_ensemble at_ensemble_t;
typedef struct {
  int64_t nsteps;
  int32_t group;
  int32_t twin;
} at_member_t;
typedef struct {
  int64_t key;                 /* group label, or the grid size n[0] */
  int32_t count;               /* members in the group */
  int32_t ntwin;               /* members of the group that have a twin */
  double rms_mean, rms_var;    /* mean and unbiased variance of the members' RMS errors */
  double abs_mean;             /* mean of the members' mean absolute errors */
  double diff_mean, diff_var;  /* mean and unbiased variance of the RMS of U - U_twin over the members with a twin */
  double dabs_mean, dabs_var;  /* the same for the mean absolute value of U - U_twin */
} at_group_stats_t;
int at_ensemble_sizes(const at_config_t *members, const at_member_t *runs, int32_t count, int64_t *ring_len,
                      int64_t *log_len);
int at_ensemble_create(const at_config_t *members, const at_member_t *runs, int32_t count, double *ring_dev,
                       int64_t ring_len, uint8_t *log_dev, int64_t log_len, int32_t threads, int32_t ctas_per_sm,
                       void *stream, at_ensemble_t **out);
int at_ensemble_run(at_ensemble_t *ens);
int at_ensemble_stats(at_ensemble_t *ens, at_stats_t *per_member, double *per_member_diff, int32_t cap,
                      at_group_stats_t *groups, int32_t gcap, int32_t *ngroups);
int at_ensemble_destroy(at_ensemble_t *ens);

/* One-line description of the last error on this thread ("" if none). */
const char *at_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ATFD_AT_H */
