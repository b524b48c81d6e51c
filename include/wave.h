/*
 * wave.h -- C ABI of libwave: memory-efficient adjoint (superposition) gradients
 * of the acoustic wave equation on one GB300 (sm_103a).
 *
 * Method: arXiv 2509.15744 (Herrmann, Buerchner, Kollmannsberger), "A Memory
 * Efficient Adjoint Method to Enable Billion Parameter Optimization on a Single
 * GPU in Dynamic Problems".  Sec. 2 states the forward problems (Eq.
 * scalarwaveequation in squared-slowness form, Eq. wavetopopt), sources
 * (Eq. source1, Eq. source2), objectives (Eq. cost1, Eq. cost2), adjoint
 * sources (Eq. adjointSource1, Eq. adjointSource2) and Frechet kernels
 * (Eq. kernel1, Eq. kernel2).  Sec. 3.1 gives the leapfrog stencils (Eq.
 * FDstencil1, Eq. FDstencil2).  Sec. 4 gives the superposed field (Eq.
 * superposedPDE, Eq. superposedforce), the approximation K~ = (K(u^s,u^s) -
 * K(u,u)) / 2k (Eq. superposedkernel) and Algorithm 1.
 *
 * General conventions
 *  - Grids are dense, C order, x fastest: cell (x, y, z) has flat index
 *    (z * ny + y) * nx + x.  In 2D nz = 1.
 *  - Pointers named *_dev are device pointers owned by the caller.  The library
 *    never allocates device memory: every call that needs scratch takes a
 *    caller workspace whose size the matching *_workspace_size call returns.
 *    Workspace must be 256-byte aligned.
 *  - All calls that take a stream enqueue their work on it and return without
 *    waiting, except where stated (wave_model_create reads back one number).
 *    Host-side validation happens before anything is enqueued; on a non-OK
 *    return nothing has been enqueued unless the status is WAVE_ECUDA.
 *  - No C++ exception crosses this boundary.  Every call returns wave_status.
 *  - The stencil state is FP32 (or BF16/FP16 storage of the resident time
 *    levels); the sensitivity accumulates in FP32 (optionally Kahan-
 *    compensated); FP64 is used only for the misfit and norm reductions.
 */
#ifndef WAVE_H
#define WAVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  WAVE_OK = 0,
  WAVE_EINVAL = 1,        /* bad argument (sizes, indices, null pointer, order) */
  WAVE_EUNSTABLE = 2,     /* dt violates the leapfrog stability bound */
  WAVE_EWORKSPACE = 3,    /* workspace too small or misaligned */
  WAVE_ECUDA = 4,         /* a CUDA runtime call failed; see wave_last_error() */
  WAVE_ETIMEOUT = 5,      /* a bounded device wait gave up */
  WAVE_ENONFINITE = 6,    /* non-finite value detected */
  WAVE_EUNSUPPORTED = 7   /* valid request this build does not implement */
} wave_status;

typedef enum {
  WAVE_VELOCITY = 0,  /* param = v [m/s]; mass m = 1/v^2, order-p Laplacian (Eq. scalarwaveequation, squared-slowness form) */
  WAVE_DENSITY = 1    /* param = gamma in [0,1]; kappa^-1, rho^-1 linear in gamma (Sec. 2.3, Eq. wavetopopt); order 2 only */
} wave_physics;

typedef enum {
  WAVE_DIRICHLET = 0, /* odd mirror about the virtual wall nodes -1 and n */
  WAVE_NEUMANN = 1    /* even mirror about the half cell (Eq. BC, ghost cells of Sec. 3.1) */
} wave_bc;

typedef enum {
  WAVE_F32 = 0,       /* resident time levels stored in FP32 */
  WAVE_BF16 = 1,      /* stored in BF16, stencil arithmetic in FP32 */
  WAVE_F16 = 2        /* stored in FP16, stencil arithmetic in FP32 */
} wave_storage;

typedef enum {
  WAVE_OBJ_L2 = 0,    /* C = 1/2 dt sum_n sum_r (u_r^n - d_r^n)^2 (Eq. cost1, rectangle rule over levels 0..N) */
  WAVE_OBJ_PATCH = 1  /* C = sign dt/n_s sum_n sum_{i in patch} (u_i^n)^2 (Eq. cost2; receivers = patch cells) */
} wave_objective;

typedef enum {
  WAVE_SUPERPOSITION = 0, /* Algorithm 1: K~ = (K(u^s,u^s) - K(u,u)) / 2k, memory independent of N */
  WAVE_EXACT_STORED = 1,  /* standard adjoint over the stored forward history (comparator; memory ~ N grids) */
  WAVE_SYMMETRIC_K = 2,   /* (K~(k) + K~(-k)) / 2 = (K(u^+,u^+) - K(u^-,u^-)) / 4k, u^+- = u +- k u_adj:
                             two superposed fields from one forward; the k^2 term of Eq. superposedkernel1
                             cancels, so the result is the exact discrete gradient (2 more grids) */
  WAVE_EXACT_REVERSE = 3  /* exact gradient without history: u reconstructed backward by time reversal
                             (leapfrog is reversible) beside the adjoint field, accumulating the mixed term
                             of Eq. kernel1 directly (velocity form, FP32 storage; 2 more grids) */
} wave_grad_mode;

typedef enum {
  WAVE_GRAD_MASS = 0,  /* dC/dm (velocity: m = 1/v^2) or dC/dgamma (density) */
  WAVE_GRAD_PARAM = 1  /* dC/dv (velocity) or dC/dgamma (density) */
} wave_grad_wrt;

/* Grid and discretisation.  n[0] = nx (fastest), n[1] = ny, n[2] = nz (1 in 2D).
 * Each axis needs n >= order + 1 cells. */
typedef struct {
  int32_t ndim;        /* 2 or 3 */
  int32_t order;       /* 2, 4, 6 or 8 (velocity); 2 (density) */
  int64_t n[3];
  double h;            /* grid spacing [m] */
  double dt;           /* time step [s] */
  int32_t physics;     /* wave_physics */
  int32_t bc;          /* wave_bc */
  int32_t storage;     /* wave_storage */
  int32_t kahan;       /* 1: Kahan-compensated sensitivity accumulation */
} wave_grid_desc;

/* One shot: a Kronecker point source (Eq. source1) and its receivers.
 * wavelet_dev: psi(t_n), t_n = n dt, n = 0..nt (sample 0 is never used).
 * rec_cells_dev: flat cell indices; an out-of-range index is skipped (its trace
 *   and residual are zero, nothing is injected there).
 * observed_dev: [nrec][nt+1] measured traces (level n at column n), or NULL
 *   for zero data (the patch objective).
 * traces_dev: [nrec][nt+1] output of wave_forward (ignored by the gradient). */
typedef struct {
  int64_t src_cell;
  int32_t nt;          /* N_s: levels 0..N_s are recorded */
  int32_t nrec;
  const float* wavelet_dev;
  const int64_t* rec_cells_dev;
  const float* observed_dev;
  float* traces_dev;
} wave_shot;

typedef struct {
  int32_t objective;   /* wave_objective */
  int32_t mode;        /* wave_grad_mode */
  int32_t batched;     /* 0: shots one after another; 1: all shots advanced together */
  int32_t grad_wrt;    /* wave_grad_wrt */
  double patch_sign;   /* +1 suppress / -1 amplify (Sec. 5.2 sign flip); patch objective only */
  double k;            /* superposition factor (Eq. superposedforce); <= 0 selects it automatically */
  double k_ratio;      /* automatic k = k_ratio * ||psi|| / ||f_adj|| of the first shot, a stand-in
                          for the calibration of Sec. 4.1 (the smallest k at which FP32 still agrees
                          with FP64); 0 -> the default: 1e-2 for WAVE_SUPERPOSITION in the velocity
                          form, 5e-2 in the density form (larger FP32 cancellation), 1 for
                          WAVE_SYMMETRIC_K (no k^2 gap) */
} wave_gradient_opts;

/* Per-call figures of a gradient call (wave_gradient_metrics_read). */
typedef struct {
  double misfit;        /* C summed over shots (Eq. cost1 / cost2), FP64 */
  double k;             /* k used (0 for WAVE_EXACT_STORED and WAVE_EXACT_REVERSE) */
  double grad_l2;       /* ||grad||_2 of the returned gradient, FP64 reduction on the device */
  double forward_ms;    /* device time of the forward pass(es), misfit and k included */
  double adjoint_ms;    /* device time of the superposed / adjoint pass(es) and the finish */
  double total_ms;      /* device time of the whole call */
  double step_bytes;    /* algorithmic bytes of the step-kernel launches (per cell and launch:
                           read u^n, u^{n-1}, coef [, b], write u^{n+1} per field, accumulator
                           [+ compensation] read-modify-write once) */
  double cell_updates;  /* sum over shots of cells x N_s: the gradient cell-updates of the call */
  int64_t step_launches;
} wave_gradient_metrics;

typedef struct wave_model_s* wave_model;

/* ---- version, errors --------------------------------------------------- */
const char* wave_status_string(wave_status s);
/* Text of the last CUDA error seen by this thread (empty if none). */
const char* wave_last_error(void);
/* Number of kernels this library has launched in this process. */
uint64_t wave_launch_count(void);

/* ---- step-kernel timing ------------------------------------------------------
 * When enabled, every launch of the fused step kernel is bracketed by CUDA
 * events on its stream.  wave_timing_read waits for the recorded events and
 * returns the summed kernel time, the number of timed launches and their
 * algorithmic bytes (per cell: read u^n, u^{n-1}, coef [+ b], write u^{n+1},
 * [+ accumulator RMW, + compensation RMW]).  Enabling resets the counters.
 * The events are recorded as external events (cudaEventRecordExternal): a
 * call captured into a CUDA graph while timing is enabled records them at
 * each replay, and wave_timing_read then returns the last replay's kernel
 * times with the launch and byte counts of the one captured call.
 * Not thread-safe. */
wave_status wave_timing_enable(int32_t on);
wave_status wave_timing_read(double* step_ms, uint64_t* step_launches, double* step_bytes);

/* ---- stability ----------------------------------------------------------
 * dt at `fraction` of the leapfrog limit for a homogeneous medium of speed
 * vmax: dt = fraction * 2h / (vmax sqrt(ndim S)), S = |c_0 + 2 sum (-1)^j c_j|
 * of the order-p central second-derivative weights (Sec. 3.1 stencil family).
 * Returns 0 on invalid input. */
double wave_cfl_dt(int32_t ndim, int32_t order, double h, double vmax, double fraction);

/* ---- source time functions ---------------------------------------------
 * Fills out_dev[0..nt] with psi(n dt).  kind 0: Ricker, (1 - 2 pi^2 f^2 tau^2)
 * exp(-pi^2 f^2 tau^2), tau = t - 1/f.  kind 1: sine burst of Eq. source2,
 * psi0 sin(w t) sin^2(w t / 2 n_c) for t <= 2 pi n_c / w, w = 2 pi f. */
wave_status wave_wavelet(int32_t kind, double freq, int32_t nc, double psi0, double dt,
                         int32_t nt, float* out_dev, void* stream);

/* ---- model ---------------------------------------------------------------
 * A model holds the per-cell coefficients derived from param (Eq. FDstencil1/2
 * prefactors) in a caller workspace of wave_model_workspace_size() bytes.
 * param_dev: dense [nz][ny][nx] FP32 (v in m/s, or gamma).  It must stay valid
 * while the model is used (the dC/dv chain rule reads it).  Create checks the
 * stability bound on the device and waits for that one number
 * (WAVE_EUNSTABLE if violated, WAVE_ENONFINITE if param holds a NaN or an
 * Inf).  Destroy frees only the host handle. */
wave_status wave_model_workspace_size(const wave_grid_desc* desc, size_t* bytes);
wave_status wave_model_create(const wave_grid_desc* desc, const float* param_dev,
                              void* workspace_dev, size_t ws_bytes, void* stream,
                              wave_model* out);
wave_status wave_model_destroy(wave_model model);
/* Tuning hook (used by the autotuner): the number of rows (2D) or planes (3D)
 * that one warp (2D) or CTA (3D) of the step kernel marches over.  Any value
 * >= 1 is valid; it changes speed, never results. */
wave_status wave_model_set_block(wave_model model, int64_t zblock);
wave_status wave_model_get_block(wave_model model, int64_t* zblock);
/* Full tiling of the 3D FP32 step kernel: zblock as above, tile_rows (8 or 16
 * rows of 128 cells per CTA), ring_depth (2 or 3 planes staged ahead) and
 * pipeline: 0: per-thread cp.async copies into a shared-memory plane ring
 * with one CTA barrier per plane (64-bit offsets: any grid size); 3: z
 * neighbours in a register queue, one cp.async-staged plane tile per plane;
 * 4: two fields of a batched launch per pass, lower z neighbours in
 * registers and upper ones from the staged tiles, 16 rows only -- the
 * default; with more than two fields and zblock <= 32 (<= 16 with Kahan
 * compensation) the accumulator tile stays in the SM's tensor memory
 * between the pairs; 5: the fields of a batched launch one after the other over
 * z-blocks of 8 planes (zblock ignored) with the accumulator of the block in
 * registers across them, the tiles copied by TMA tensor copies into an
 * mbarrier ring that holds one field's tiles, 16 rows only.  Pipelines 3-5
 * send a launch of one field to the register-queue kernel.  Speed only;
 * results are identical. */
wave_status wave_model_set_tiling(wave_model model, int64_t zblock, int32_t tile_rows, int32_t ring_depth,
                                  int32_t pipeline);
/* Launch order of the CTAs of the 3D FP32 step kernels, pipelines 3 and 4
 * (speed only; results are bitwise the same).  cta_order 0: the CTAs of one
 * x strip and y tile launch z-block after z-block; 1 (the default):
 * plane-major, the x strips and then the y tiles of one z-block launch next to
 * each other, so the CTAs whose staged halo rows overlap run at the same time
 * and read those rows from L2 rather than HBM.  It matters once the CTAs of
 * one z-block outnumber the resident ones (1024^3 with z-blocks of 16
 * planes: 3.4% less time per launch).  A grid of more than 65535 z-blocks
 * launches in order 0 whatever the setting.  Other values: WAVE_EINVAL. */
wave_status wave_model_set_schedule(wave_model model, int32_t cta_order);
/* Waits for `stream` and reports whether a bounded device wait of a step
 * kernel gave up since the last check (WAVE_ETIMEOUT; the results of that
 * call are invalid; the error word is cleared), else whether the parameter of
 * the last wave_model_set_param (or create) breaks the stability bound
 * (WAVE_EUNSTABLE) or holds a NaN or Inf (WAVE_ENONFINITE). */
wave_status wave_model_check(wave_model model, void* stream);
/* New parameter values for an existing model (e.g. one optimisation step):
 * recomputes the coefficients and the stability maximum on `stream` without
 * waiting (wave_model_check reports the outcome).  param_dev: dense FP32 grid
 * of the model's shape; it replaces the create-time param (also for the dC/dv
 * chain rule) and must stay valid while the model is used. */
wave_status wave_model_set_param(wave_model model, const float* param_dev, void* stream);
/* Test hook: stall_pipeline = 1 makes the TMA-tiled pipeline issue no copies, so
 * its first wait runs out after wait_limit_cycles (default about 4e9 cycles);
 * used to test the time-out path without a hang.  Not for production use. */
wave_status wave_model_set_debug(wave_model model, int32_t stall_pipeline, int64_t wait_limit_cycles);

/* Row pitch (cells) of the model's resident grids: nx rounded up to 128.
 * A pitched grid is [nz][ny][pitch] FP32 (or 16-bit storage), padding zero. */
wave_status wave_model_pitch(wave_model model, int64_t* pitch);

/* ---- one step ----------------------------------------------------------------
 * One leapfrog step (Eq. FDstencil1 / FDstencil2 without force) of nfields
 * independent fields on this model, in the launch configuration of the
 * batched gradient (3D velocity form, FP32 storage: all fields in one launch;
 * otherwise one launch per field):
 *   prev_dev[f] <- 2 cur_dev[f] - prev_dev[f] + dt^2/a L cur_dev[f]
 * and, if acc_dev is not NULL, the sensitivity increment of Algorithm 1 for
 * that step: acc += acc_sign[f] * (u^{n+1} - u^n)^2 (density form: da times
 * that minus dbs times the face-weighted squared differences of u^n), with
 * Kahan compensation in comp_dev if not NULL.
 * cur_dev, prev_dev: host arrays of nfields device pointers, each a pitched
 * grid of the model's storage type, 16-byte aligned; prev_dev[f] is
 * overwritten.  acc_sign: host array of nfields factors (NULL: all +1).
 * acc_dev, comp_dev: pitched FP32 grids.  nfields in 1..32.  Asynchronous on
 * stream. */
wave_status wave_step(wave_model model, int32_t nfields, const void* const* cur_dev, void* const* prev_dev,
                      const float* acc_sign, float* acc_dev, float* comp_dev, void* stream);

/* ---- forward ---------------------------------------------------------------
 * Leapfrog u^{n+1} = 2u^n - u^{n-1} + dt^2/a (L u^n + f^n) for n = 1..N_s with
 * traces of levels 0..N_s written to each shot's traces_dev.
 * init_dev: NULL for u^0 = u^1 = 0 (Eq. IC), else dense {u^0, u^1} (2 grids).
 * final_dev: NULL, or dense output {u^N, u^{N+1}} of the last shot. */
wave_status wave_forward_workspace_size(wave_model model, const wave_shot* shots, int32_t nshots,
                                        size_t* bytes);
wave_status wave_forward(wave_model model, const wave_shot* shots, int32_t nshots,
                         const float* init_dev, float* final_dev,
                         void* workspace_dev, size_t ws_bytes, void* stream);

/* ---- gradient (Algorithm 1) -----------------------------------------------
 * Superposition mode: per shot, forward N_s steps (plus one unrecorded step to
 * N_s + 1) accumulating -K(u,u), form the adjoint source f_adj^n = -w (u_r^n -
 * d_r^n) (Eq. adjointSource1/2), then run the superposed field u^s = u + k u_adj
 * backward from (u^{N+1}, u^N) with force f + k f_adj (Eq. superposedforce)
 * accumulating +K(u^s,u^s); K~ = difference / 2k (Eq. superposedkernel).
 * grad_dev: dense FP32 grid, summed over shots, w.r.t. opts->grad_wrt.
 * misfit_dev: one double, C summed over shots.  k_dev: one double, the k used
 * (all shots share it).  grad_norm_dev: NULL or one double receiving
 * ||grad_dev||_2, reduced in FP64 on the device by the finish pass
 * (deterministic: fixed partial sums in a fixed order).  Exact mode (velocity form, FP32 storage, one shot at
 * a time) stores the forward history u^0..u^{N+1} instead and returns the
 * standard adjoint gradient; k_dev then receives 0.
 * WAVE_SYMMETRIC_K: the forward accumulates nothing; two superposed fields
 * with +k and -k run backward from copies of (u^{N+1}, u^N), accumulating
 * -K(u^+,u^+) and +K(u^-,u^-); the result is divided by 4k.  In 3D velocity
 * form with FP32 storage both fields advance in one launch (coef and the
 * accumulator are read once per step).
 * WAVE_EXACT_REVERSE: per backward step j, u^{j-1} = 2u^j - u^{j+1} + dt^2/m
 * (L u^j + f^j) and the adjoint lambda^{j-1} from lambda^{N+1} = lambda^N = 0
 * with the adjoint source alone, accumulating -(lambda^j - lambda^{j-1})
 * (u^j - u^{j-1}); k_dev receives 0.  Neither new mode supports batched = 1. */
wave_status wave_gradient_workspace_size(wave_model model, const wave_shot* shots, int32_t nshots,
                                         const wave_gradient_opts* opts, size_t* bytes);
wave_status wave_adjoint_sensitivity(wave_model model, const wave_shot* shots, int32_t nshots,
                                     const wave_gradient_opts* opts, float* grad_dev,
                                     double* misfit_dev, double* k_dev, double* grad_norm_dev,
                                     void* workspace_dev, size_t ws_bytes, void* stream);

/* ---- per-call metrics --------------------------------------------------------
 * wave_model_set_metrics(model, 1) makes every later gradient call on the model
 * record CUDA events at its pass boundaries (forward, superposed / adjoint,
 * finish) on its stream; 0 (the default) records nothing.  Not for use while
 * the stream is being captured into a CUDA graph.
 * wave_gradient_metrics_read waits for the last gradient call on the model and
 * fills *out: C, k, ||grad||_2 (the FP64 device reduction of the finish pass),
 * device times per pass, the algorithmic bytes of the step launches and the
 * cell-updates.  The call's workspace must not have been reused since.
 * Returns WAVE_EINVAL when metrics are off or no call was recorded, and
 * WAVE_ENONFINITE (after filling *out) when C, k or ||grad|| is not finite:
 * the optional end-of-call check for NaN or Inf results. */
wave_status wave_model_set_metrics(wave_model model, int32_t on);
wave_status wave_gradient_metrics_read(wave_model model, wave_gradient_metrics* out);

/* ---- misfit ----------------------------------------------------------------
 * out_dev[0] = 0.5 * weight * dt * sum_i (syn_i - obs_i)^2 in FP64 over count
 * FP32 samples (Eq. cost1 with the rectangle rule); obs_dev may be NULL (zero).
 * Deterministic two-pass reduction through caller scratch of
 * wave_misfit_scratch_size(count) bytes. */
size_t wave_misfit_scratch_size(int64_t count);
wave_status misfit(const float* syn_dev, const float* obs_dev, int64_t count, double dt,
                   double weight, double* out_dev, void* scratch_dev, size_t scratch_bytes,
                   void* stream);

/* ---- misfit without caller scratch ----------------------------------------
 * The paper has no counterpart: this is a library convenience.  Same result as
 * misfit() (FP64, within rounding of the summation order) for callers that
 * cannot allocate device memory -- e.g. a plugin whose host framework has
 * reserved all device memory for its own allocator, or a latency-critical loop
 * that must not enter an allocator.  The partial sums live in a static device
 * array inside the library (32 KB per GPU that loads it, held until exit), so
 * count is limited to 33,554,432 samples; larger counts return WAVE_EINVAL
 * before any work is enqueued.  Allocates nothing.  All calls on a GPU share
 * the array: calls whose kernels may overlap on the GPU (e.g. on unordered
 * streams) race and must not be issued.  The first call on a device looks up
 * the array's address (cudaGetSymbolAddress, with that device current) and
 * caches it with the device's context (a call in a new context after a
 * device reset looks it up again); make the first call before any stream
 * capture starts.  WAVE_ECUDA leaves the failing call's text in
 * wave_last_error(). */
wave_status wave_misfit_static(const float* syn_dev, const float* obs_dev, int64_t count, double dt,
                               double weight, double* out_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* WAVE_H */
