// Host side of libwave: argument validation, workspace carving and the time
// loop of Algorithm 1 (Sec. 4) over the fused kernels.  All work is enqueued
// on the caller's stream; the only host wait is the stability check of
// wave_model_create.  No device memory is allocated here.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "wave_internal.cuh"

using namespace wave;

namespace wave {
uint64_t launches();
}

static thread_local std::string g_last_error;
static thread_local std::string g_inner_error;   // the failing call inside a launcher, if it said

void wave::set_last_error(const char* what, cudaError_t e) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
}

void wave::note_error(const char* what, cudaError_t e) {
  g_inner_error = std::string(what) + ": " + cudaGetErrorString(e);
}

#define CUDA_TRY(expr)                                                            \
  do {                                                                            \
    g_inner_error.clear();                                                        \
    cudaError_t _e = (expr);                                                      \
    if (_e != cudaSuccess) {                                                      \
      g_last_error = std::string(#expr) + ": " + cudaGetErrorString(_e);          \
      if (!g_inner_error.empty()) g_last_error += " (in " + g_inner_error + ")"; \
      return WAVE_ECUDA;                                                          \
    }                                                                             \
  } while (0)

// ---------------------------------------------------------------------------
// workspace carving: the same walk computes sizes (base == nullptr) and
// pointers, 256-byte aligned.
// ---------------------------------------------------------------------------
struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(void* b) : base(static_cast<char*>(b)) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
  void* take_bytes(size_t bytes) { return take<char>(bytes); }
};

static size_t storage_bytes(int storage) { return storage == WAVE_F32 ? 4 : 2; }

// Central second-derivative weights c_0..c_r (Sec. 3.1 family, textbook values).
static const double kWeights[4][5] = {
    {-2.0, 1.0, 0, 0, 0},
    {-5.0 / 2.0, 4.0 / 3.0, -1.0 / 12.0, 0, 0},
    {-49.0 / 18.0, 3.0 / 2.0, -3.0 / 20.0, 1.0 / 90.0, 0},
    {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0}};

static double symbol_max(int order) {
  const int r = order / 2;
  double s = kWeights[r - 1][0];
  for (int j = 1; j <= r; ++j) s += 2.0 * ((j & 1) ? -1.0 : 1.0) * kWeights[r - 1][j];
  return fabs(s);
}

// Material derivatives of the acoustic model (Sec. 2.3).
static const double kDa = 1.0 / 6.87e8 - 1.0 / 1.419e5;   // d kappa^-1 / d gamma
static const double kDb = 1.0 / 2643.0 - 1.0 / 1.204;     // d rho^-1 / d gamma

struct wave_model_s {
  wave_grid_desc d;
  Geom g;
  const float* param;
  float* coef;
  float* bmat;
  int64_t zblock;
  int tile_rows;     // 3D ring kernel: 8 or 16 rows per CTA
  int ring_depth;    // 3D ring kernel: 2 or 3 planes copied ahead
  int pipeline;      // 3D FP32: 0 cp.async ring (any size), 3 register queue in z + staged plane tiles,
                     // 4 as 3 with two shots per pass (batched), 5 as 4 with TMA tensor tiles
  int cta_order;     // 3D pipelines 3, 4: 0 z-block fastest, 1 plane-major launch order
  int* err;          // device error word (bounded waits)
  float* part;       // stability partial maxima
  float* maxv;       // stability: max over cells of (v dt / h)^2 S-scaled (<= 4 is stable)
  double sym;        // the operator's symbol scale used by the stability kernel
  long long wait_limit_cycles;
  int debug_stall;
  double stability;
  // per-call metrics (wave_model_set_metrics): CUDA events at the pass
  // boundaries of the last gradient call and where its device scalars live
  struct Metrics {
    bool on = false;
    bool valid = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> kind;      // kEv* of each recorded event
    size_t used = 0;
    double bytes = 0.0;         // algorithmic bytes of the step launches
    double units = 0.0;         // sum_s ncells * N_s
    uint64_t launches = 0;
    const double* scal = nullptr;   // [0] k, [4] sum grad^2, [6] C
    int mode = 0;
  };
  mutable Metrics met;
};

// Records a timing event on s.  While s is being captured into a CUDA graph
// the event is recorded as an external event node, so every replay records
// it; outside capture that flag is not allowed and a plain record is used.
static cudaError_t record_event(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t err = cudaStreamIsCapturing(s, &cs);
  if (err != cudaSuccess) return err;
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                                             : cudaEventRecord(e, s);
}

enum { kEvStart = 0, kEvForwardEnd = 1, kEvAdjointEnd = 2 };

// Record a pass boundary of the current gradient call (metrics on only).
static cudaError_t mark(const wave_model_s* m, int kind, cudaStream_t s) {
  auto& M = m->met;
  if (!M.on) return cudaSuccess;
  if (M.used == M.ev.size()) {
    cudaEvent_t e;
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return err;
    M.ev.push_back(e);
  }
  if (M.kind.size() <= M.used) M.kind.resize(M.used + 1);
  M.kind[M.used] = kind;
  return record_event(M.ev[M.used++], s);
}

static wave_status validate_desc(const wave_grid_desc* d) {
  if (!d) return WAVE_EINVAL;
  if (d->ndim != 2 && d->ndim != 3) return WAVE_EINVAL;
  if (d->order != 2 && d->order != 4 && d->order != 6 && d->order != 8) return WAVE_EINVAL;
  if (d->physics != WAVE_VELOCITY && d->physics != WAVE_DENSITY) return WAVE_EINVAL;
  if (d->bc != WAVE_DIRICHLET && d->bc != WAVE_NEUMANN) return WAVE_EINVAL;
  if (d->storage < WAVE_F32 || d->storage > WAVE_F16) return WAVE_EINVAL;
  if (!(d->h > 0.0) || !(d->dt > 0.0)) return WAVE_EINVAL;
  for (int a = 0; a < d->ndim; ++a)
    if (d->n[a] < d->order + 1) return WAVE_EINVAL;
  if (d->ndim == 2 && d->n[2] != 1) return WAVE_EINVAL;
  if (d->physics == WAVE_DENSITY && d->order != 2) return WAVE_EINVAL;
  return WAVE_OK;
}

static Geom make_geom(const wave_grid_desc* d) {
  Geom g;
  g.ndim = d->ndim;
  g.r = d->order / 2;
  g.bc = d->bc;
  g.nx = d->n[0];
  g.ny = d->n[1];
  g.nz = d->ndim == 3 ? d->n[2] : 1;
  g.px = (g.nx + kStrip - 1) / kStrip * kStrip;
  g.plane = g.px * g.ny;
  g.cells = g.plane * g.nz;
  return g;
}

static int64_t default_zblock(const Geom& g, bool kahan) {
  const int64_t nstrips = (g.nx + kStrip - 1) / kStrip;
  if (g.ndim == 2) {
    // about 24 warps per SM over 152 SMs
    int64_t by = nstrips * g.ny / (152 * 24);
    return std::max<int64_t>(8, std::min<int64_t>(by, 256));
  }
  // the largest z-block whose accumulator tile (and compensation) fits the
  // tensor memory of the batched two-shots-per-pass kernel
  return std::min<int64_t>(kahan ? 16 : 32, g.nz);
}

extern "C" {

const char* wave_status_string(wave_status s) {
  switch (s) {
    case WAVE_OK: return "ok";
    case WAVE_EINVAL: return "invalid argument";
    case WAVE_EUNSTABLE: return "time step violates the leapfrog stability bound";
    case WAVE_EWORKSPACE: return "workspace too small or misaligned";
    case WAVE_ECUDA: return "CUDA error";
    case WAVE_ETIMEOUT: return "bounded device wait timed out";
    case WAVE_ENONFINITE: return "non-finite value";
    case WAVE_EUNSUPPORTED: return "not supported by this build";
  }
  return "unknown status";
}

const char* wave_last_error(void) { return g_last_error.c_str(); }

uint64_t wave_launch_count(void) { return wave::launches(); }

double wave_cfl_dt(int32_t ndim, int32_t order, double h, double vmax, double fraction) {
  if ((ndim != 2 && ndim != 3 && ndim != 1) || (order != 2 && order != 4 && order != 6 && order != 8)) return 0.0;
  if (!(h > 0) || !(vmax > 0) || !(fraction > 0)) return 0.0;
  return fraction * 2.0 * h / (vmax * sqrt(ndim * symbol_max(order)));
}

wave_status wave_wavelet(int32_t kind, double freq, int32_t nc, double psi0, double dt, int32_t nt, float* out_dev,
                         void* stream) {
  if ((kind != 0 && kind != 1) || !(freq > 0) || !(dt > 0) || nt < 0 || !out_dev) return WAVE_EINVAL;
  if (kind == 1 && nc < 1) return WAVE_EINVAL;
  CUDA_TRY(launch_wavelet(kind, freq, nc, psi0, dt, nt, out_dev, (cudaStream_t)stream));
  return WAVE_OK;
}

// ---------------------------------------------------------------------------
// model
// ---------------------------------------------------------------------------
static void carve_model(Carve& c, const Geom& g, int physics, float** coef, float** bmat, float** part,
                        float** maxv, int** err) {
  *coef = c.take<float>(g.cells);
  *bmat = physics == WAVE_DENSITY ? c.take<float>(g.cells) : nullptr;
  *part = c.take<float>(1024);
  *maxv = c.take<float>(1);
  *err = c.take<int>(1);
}

wave_status wave_model_workspace_size(const wave_grid_desc* desc, size_t* bytes) {
  wave_status st = validate_desc(desc);
  if (st != WAVE_OK) return st;
  if (!bytes) return WAVE_EINVAL;
  Geom g = make_geom(desc);
  Carve c(nullptr);
  float *a, *b, *p, *m;
  int* e;
  carve_model(c, g, desc->physics, &a, &b, &p, &m, &e);
  *bytes = c.off;
  return WAVE_OK;
}

wave_status wave_model_create(const wave_grid_desc* desc, const float* param_dev, void* workspace_dev,
                              size_t ws_bytes, void* stream, wave_model* out) {
  wave_status st = validate_desc(desc);
  if (st != WAVE_OK) return st;
  if (!param_dev || !out || !workspace_dev) return WAVE_EINVAL;
  if (reinterpret_cast<uintptr_t>(workspace_dev) % 256) return WAVE_EWORKSPACE;
  size_t need = 0;
  wave_model_workspace_size(desc, &need);
  if (ws_bytes < need) return WAVE_EWORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  Geom g = make_geom(desc);
  Carve c(workspace_dev);
  float *coef, *bmat, *part, *maxv;
  int* errw;
  carve_model(c, g, desc->physics, &coef, &bmat, &part, &maxv, &errw);
  CUDA_TRY(cudaMemsetAsync(errw, 0, sizeof(int), s));
  double sym;
  if (desc->physics == WAVE_VELOCITY) {
    CUDA_TRY(launch_coef_velocity(g, param_dev, (float)(desc->dt / desc->h), coef, s));
    sym = desc->ndim * symbol_max(desc->order);
  } else {
    CUDA_TRY(launch_coef_density(g, param_dev, desc->dt * desc->dt / (desc->h * desc->h), coef, bmat, s));
    sym = 0.0;
  }
  const int nparts = 1024;
  CUDA_TRY(launch_stability(g, desc->physics, sym, coef, bmat, part, nparts, s));
  CUDA_TRY(launch_max_final(part, nparts, maxv, s));
  float host_max = 0.f;
  CUDA_TRY(cudaMemcpyAsync(&host_max, maxv, sizeof(float), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (!isfinite(host_max)) return WAVE_ENONFINITE;   // a NaN or Inf parameter
  if (!(host_max <= 4.0f * (1.0f + 1e-5f))) return WAVE_EUNSTABLE;
  wave_model_s* m = new wave_model_s;
  m->d = *desc;
  m->g = g;
  m->param = param_dev;
  m->coef = coef;
  m->bmat = bmat;
  m->zblock = default_zblock(g, desc->kahan != 0);
  // untuned default: one field per launch on the register-queue kernel, two
  // or more on the two-shots-per-pass kernel (the faster of the batched ones
  // on every measured workload)
  m->tile_rows = 16;
  m->ring_depth = 2;
  m->pipeline = 4;
  m->cta_order = 1;
  m->err = errw;
  m->part = part;
  m->maxv = maxv;
  m->sym = sym;
  m->wait_limit_cycles = 4000000000LL;  // about two seconds at the maximum SM clock
  m->debug_stall = 0;
  m->stability = host_max;
  *out = m;
  return WAVE_OK;
}

wave_status wave_model_destroy(wave_model model) {
  if (model)
    for (cudaEvent_t e : model->met.ev) cudaEventDestroy(e);
  delete model;
  return WAVE_OK;
}

// Tuning hook: rows (2D) or planes (3D) that one warp / CTA marches over.
wave_status wave_model_set_block(wave_model model, int64_t zblock) {
  if (!model || zblock < 1) return WAVE_EINVAL;
  model->zblock = zblock;
  return WAVE_OK;
}

wave_status wave_model_get_block(wave_model model, int64_t* zblock) {
  if (!model || !zblock) return WAVE_EINVAL;
  *zblock = model->zblock;
  return WAVE_OK;
}

wave_status wave_model_set_tiling(wave_model model, int64_t zblock, int32_t tile_rows, int32_t ring_depth,
                                  int32_t pipeline) {
  if (!model || zblock < 1) return WAVE_EINVAL;
  if (tile_rows != 8 && tile_rows != 16) return WAVE_EINVAL;
  if (ring_depth != 2 && ring_depth != 3) return WAVE_EINVAL;
  if (pipeline != 0 && (pipeline < 3 || pipeline > 5)) return WAVE_EINVAL;
  if ((pipeline == 4 || pipeline == 5) && tile_rows != 16) return WAVE_EINVAL;
  model->zblock = zblock;
  model->tile_rows = tile_rows;
  model->ring_depth = ring_depth;
  model->pipeline = pipeline;
  return WAVE_OK;
}

wave_status wave_model_set_schedule(wave_model model, int32_t cta_order) {
  if (!model) return WAVE_EINVAL;
  if (cta_order != 0 && cta_order != 1) return WAVE_EINVAL;
  model->cta_order = cta_order;
  return WAVE_OK;
}

wave_status wave_model_check(wave_model model, void* stream) {
  if (!model) return WAVE_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int host = 0;
  float mx = 0.f;
  CUDA_TRY(cudaMemcpyAsync(&host, model->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(&mx, model->maxv, sizeof(float), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (host) {
    CUDA_TRY(cudaMemsetAsync(model->err, 0, sizeof(int), s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return WAVE_ETIMEOUT;
  }
  if (!isfinite(mx)) return WAVE_ENONFINITE;
  if (!(mx <= 4.0f * (1.0f + 1e-5f))) return WAVE_EUNSTABLE;
  return WAVE_OK;
}

// New parameter values for an existing model (an optimisation step): the
// coefficients and the stability maximum are recomputed on the stream with no
// host wait; wave_model_check reports an unstable or non-finite parameter.
wave_status wave_model_set_param(wave_model m, const float* param_dev, void* stream) {
  if (!m || !param_dev) return WAVE_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const wave_grid_desc* desc = &m->d;
  if (desc->physics == WAVE_VELOCITY)
    CUDA_TRY(launch_coef_velocity(m->g, param_dev, (float)(desc->dt / desc->h), m->coef, s));
  else
    CUDA_TRY(launch_coef_density(m->g, param_dev, desc->dt * desc->dt / (desc->h * desc->h), m->coef, m->bmat, s));
  const int nparts = 1024;
  CUDA_TRY(launch_stability(m->g, desc->physics, m->sym, m->coef, m->bmat, m->part, nparts, s));
  CUDA_TRY(launch_max_final(m->part, nparts, m->maxv, s));
  m->param = param_dev;
  return WAVE_OK;
}

wave_status wave_model_set_debug(wave_model model, int32_t stall_pipeline, int64_t wait_limit_cycles) {
  if (!model || wait_limit_cycles < 1) return WAVE_EINVAL;
  model->debug_stall = stall_pipeline != 0;
  model->wait_limit_cycles = wait_limit_cycles;
  return WAVE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// shared pieces of the time loops
// ---------------------------------------------------------------------------
static wave_status validate_shots(const wave_model_s* m, const wave_shot* shots, int32_t nshots, bool need_traces) {
  if (!shots || nshots < 1) return WAVE_EINVAL;
  const int64_t total = m->g.nx * m->g.ny * m->g.nz;
  for (int s = 0; s < nshots; ++s) {
    const wave_shot& sh = shots[s];
    if (sh.nt < 1 || sh.nrec < 0) return WAVE_EINVAL;
    if (sh.src_cell < 0 || sh.src_cell >= total) return WAVE_EINVAL;
    if (!sh.wavelet_dev) return WAVE_EINVAL;
    if (sh.nrec > 0 && !sh.rec_cells_dev) return WAVE_EINVAL;
    if (need_traces && sh.nrec > 0 && !sh.traces_dev) return WAVE_EINVAL;
  }
  return WAVE_OK;
}

static int64_t pitched_cell(const Geom& g, int64_t flat) { return (flat / g.nx) * g.px + flat % g.nx; }

static StepArgs step_args(const wave_model_s* m, const void* cur, void* prev) {
  StepArgs a;
  memset(&a, 0, sizeof(a));
  a.g = m->g;
  a.u_cur = cur;
  a.u_prev = prev;
  a.coef = m->coef;
  a.bmat = m->bmat;
  a.da = m->d.physics == WAVE_DENSITY ? (float)kDa : 1.f;
  a.dbs = m->d.physics == WAVE_DENSITY ? (float)(m->d.dt * m->d.dt / (m->d.h * m->d.h) * kDb) : 0.f;
  a.zblock = m->zblock;
  a.tile_rows = m->tile_rows;
  a.ring_depth = m->ring_depth;
  a.pipeline = m->pipeline;
  a.cta_order = m->cta_order;
  a.err = m->err;
  a.wait_limit_cycles = m->wait_limit_cycles;
  a.debug_stall = m->debug_stall;
  return a;
}

// ---- optional per-launch timing of the step kernel (CUDA events on the
// launching stream), read back by wave_timing_read.  The events are recorded
// as external events, so a gradient call captured into a CUDA graph records
// them at every replay (the last replay's times are read) -------------------
struct StepTiming {
  bool on = false;
  std::vector<cudaEvent_t> ev;
  size_t used = 0;
  double bytes = 0.0;      // algorithmic bytes of the timed launches
  uint64_t launches = 0;
};
static StepTiming g_timing;


static double step_bytes(const wave_model_s* m, const StepArgs& a) {
  const double cells = (double)(m->g.nx * m->g.ny * m->g.nz);
  const double eb = (double)storage_bytes(m->d.storage);
  double b = 3.0 * eb + 4.0;                    // read u^n, u^{n-1}, coef; write u^{n+1}
  if (m->d.physics == WAVE_DENSITY) b += 4.0;   // read b
  if (a.acc_mass || a.acc_stiff) b += a.comp ? 16.0 : 8.0;  // accumulator (+ compensation) RMW
  return cells * b;
}

static cudaError_t run_step(const wave_model_s* m, const StepArgs& a, cudaStream_t s) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (g_timing.on) {
    while (g_timing.ev.size() < g_timing.used + 2) {
      cudaEvent_t e;
      cudaError_t err = cudaEventCreate(&e);
      if (err != cudaSuccess) return err;
      g_timing.ev.push_back(e);
    }
    e0 = g_timing.ev[g_timing.used];
    e1 = g_timing.ev[g_timing.used + 1];
    g_timing.used += 2;
    cudaError_t err = record_event(e0, s);
    if (err != cudaSuccess) return err;
  }
  cudaError_t err = m->d.physics == WAVE_VELOCITY ? launch_step_velocity(a, m->d.order, m->d.storage, s)
                                                  : launch_step_density(a, m->d.storage, s);
  if (err != cudaSuccess) return err;
  if (g_timing.on) {
    err = record_event(e1, s);
    g_timing.bytes += step_bytes(m, a);
    g_timing.launches += 1;
  }
  if (m->met.on) {
    m->met.bytes += step_bytes(m, a);
    m->met.launches += 1;
  }
  return err;
}

static cudaError_t run_batched(const wave_model_s* m, const BatchArgs& b, cudaStream_t s) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (g_timing.on) {
    while (g_timing.ev.size() < g_timing.used + 2) {
      cudaEvent_t e;
      cudaError_t err = cudaEventCreate(&e);
      if (err != cudaSuccess) return err;
      g_timing.ev.push_back(e);
    }
    e0 = g_timing.ev[g_timing.used];
    e1 = g_timing.ev[g_timing.used + 1];
    g_timing.used += 2;
    cudaError_t err = record_event(e0, s);
    if (err != cudaSuccess) return err;
  }
  cudaError_t err = launch_step3d_batched(b, m->d.order, s);
  if (err != cudaSuccess) return err;
  const double cells = (double)(m->g.nx * m->g.ny * m->g.nz);
  bool any = false;
  for (int i = 0; i < b.nshots; ++i) any |= b.accf[i] != 0;
  // per shot: read u^n, u^{n-1}, write u^{n+1}; once: coef, acc (+comp) RMW
  const double bytes = cells * (12.0 * b.nshots + 4.0 + (any ? (b.base.comp ? 16.0 : 8.0) : 0.0));
  if (g_timing.on) {
    err = record_event(e1, s);
    g_timing.bytes += bytes;
    g_timing.launches += 1;
  }
  if (m->met.on) {
    m->met.bytes += bytes;
    m->met.launches += 1;
  }
  return err;
}

extern "C" wave_status wave_timing_enable(int32_t on) {
  g_timing.on = on != 0;
  g_timing.used = 0;
  g_timing.bytes = 0.0;
  g_timing.launches = 0;
  return WAVE_OK;
}

extern "C" wave_status wave_timing_read(double* step_ms, uint64_t* step_launches, double* step_bytes_total) {
  if (!step_ms || !step_launches || !step_bytes_total) return WAVE_EINVAL;
  double total = 0.0;
  for (size_t i = 0; i + 1 < g_timing.used; i += 2) {
    CUDA_TRY(cudaEventSynchronize(g_timing.ev[i + 1]));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, g_timing.ev[i], g_timing.ev[i + 1]));
    total += ms;
  }
  *step_ms = total;
  *step_launches = g_timing.launches;
  *step_bytes_total = g_timing.bytes;
  return WAVE_OK;
}

static SparseArgs sparse_args(const wave_model_s* m, const int64_t* recp, int32_t nrec) {
  SparseArgs a;
  memset(&a, 0, sizeof(a));
  a.rec_p = recp;
  a.nrec = nrec;
  a.glevel = -1;
  a.src_p = -1;
  a.ilevel = 0;
  a.coef = m->coef;
  a.h2 = (float)(m->d.h * m->d.h);
  a.inj_sign = -1.f;
  return a;
}

extern "C" wave_status wave_model_pitch(wave_model m, int64_t* pitch) {
  if (!m || !pitch) return WAVE_EINVAL;
  *pitch = m->g.px;
  return WAVE_OK;
}

// ---------------------------------------------------------------------------
// one step of several fields (the step of Algorithm 1's loops, no force)
// ---------------------------------------------------------------------------
extern "C" wave_status wave_step(wave_model m, int32_t nfields, const void* const* cur_dev, void* const* prev_dev,
                                 const float* acc_sign, float* acc_dev, float* comp_dev, void* stream) {
  if (!m || !cur_dev || !prev_dev || nfields < 1 || nfields > kMaxBatch) return WAVE_EINVAL;
  if (comp_dev && !acc_dev) return WAVE_EINVAL;
  auto misaligned = [](const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 != 0; };
  if (misaligned(acc_dev) || misaligned(comp_dev)) return WAVE_EINVAL;
  for (int f = 0; f < nfields; ++f) {
    if (!cur_dev[f] || !prev_dev[f] || misaligned(cur_dev[f]) || misaligned(prev_dev[f])) return WAVE_EINVAL;
    if (cur_dev[f] == prev_dev[f]) return WAVE_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const bool one_launch = m->d.ndim == 3 && m->d.physics == WAVE_VELOCITY && m->d.storage == WAVE_F32;
  if (one_launch) {
    BatchArgs b;
    memset(&b, 0, sizeof(b));
    b.base = step_args(m, nullptr, nullptr);
    b.base.acc = acc_dev;
    b.base.comp = comp_dev;
    b.base.acc_scale = 1.f;
    b.err = m->err;
    b.wait_limit_cycles = m->wait_limit_cycles;
    b.debug_stall = m->debug_stall;
    b.nshots = nfields;
    for (int f = 0; f < nfields; ++f) {
      b.cur[f] = static_cast<const float*>(cur_dev[f]);
      b.prev[f] = static_cast<float*>(prev_dev[f]);
      b.accf[f] = acc_dev ? (acc_sign ? acc_sign[f] : 1.f) : 0.f;
    }
    CUDA_TRY(run_batched(m, b, s));
    return WAVE_OK;
  }
  for (int f = 0; f < nfields; ++f) {
    StepArgs a = step_args(m, cur_dev[f], prev_dev[f]);
    const float sg = acc_sign ? acc_sign[f] : 1.f;
    if (acc_dev && sg != 0.f) {
      a.acc = acc_dev;
      a.comp = comp_dev;
      a.acc_scale = sg;
      a.acc_mass = 1;
      a.acc_stiff = 1;
    }
    CUDA_TRY(run_step(m, a, s));
  }
  return WAVE_OK;
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
static void carve_forward(Carve& c, const wave_model_s* m, const wave_shot* shots, int32_t nshots, void** u0,
                          void** u1, int64_t** recp) {
  int32_t maxrec = 1;
  for (int s = 0; s < nshots; ++s) maxrec = std::max(maxrec, shots[s].nrec);
  const size_t eb = storage_bytes(m->d.storage);
  *u0 = c.take_bytes(m->g.cells * eb);
  *u1 = c.take_bytes(m->g.cells * eb);
  *recp = c.take<int64_t>(maxrec);
}

extern "C" wave_status wave_forward_workspace_size(wave_model m, const wave_shot* shots, int32_t nshots,
                                                   size_t* bytes) {
  if (!m || !bytes) return WAVE_EINVAL;
  wave_status st = validate_shots(m, shots, nshots, false);
  if (st != WAVE_OK) return st;
  Carve c(nullptr);
  void *u0, *u1;
  int64_t* recp;
  carve_forward(c, m, shots, nshots, &u0, &u1, &recp);
  *bytes = c.off;
  return WAVE_OK;
}

extern "C" wave_status wave_forward(wave_model m, const wave_shot* shots, int32_t nshots, const float* init_dev,
                                    float* final_dev, void* ws, size_t ws_bytes, void* stream) {
  if (!m) return WAVE_EINVAL;
  wave_status st = validate_shots(m, shots, nshots, true);
  if (st != WAVE_OK) return st;
  size_t need = 0;
  wave_forward_workspace_size(m, shots, nshots, &need);
  if (!ws || ws_bytes < need || reinterpret_cast<uintptr_t>(ws) % 256) return WAVE_EWORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const Geom& g = m->g;
  const int stor = m->d.storage;
  const size_t eb = storage_bytes(stor);
  Carve c(ws);
  void *ua, *ub;
  int64_t* recp;
  carve_forward(c, m, shots, nshots, &ua, &ub, &recp);
  const int64_t ncells = g.nx * g.ny * g.nz;
  for (int si = 0; si < nshots; ++si) {
    const wave_shot& sh = shots[si];
    const int N = sh.nt;
    CUDA_TRY(launch_pitch_indices(g, sh.rec_cells_dev, sh.nrec, recp, s));
    if (init_dev) {
      CUDA_TRY(launch_dense_to_pitched(g, init_dev, ua, stor, s));
      CUDA_TRY(launch_dense_to_pitched(g, init_dev + ncells, ub, stor, s));
    } else {
      CUDA_TRY(cudaMemsetAsync(ua, 0, g.cells * eb, s));
      CUDA_TRY(cudaMemsetAsync(ub, 0, g.cells * eb, s));
    }
    SparseArgs sp = sparse_args(m, recp, sh.nrec);
    sp.traces = sh.traces_dev;
    sp.tr_ld = N + 1;
    sp.gsrc = ua;
    sp.glevel = 0;
    CUDA_TRY(launch_sparse(sp, stor, s));
    sp.gsrc = ub;
    sp.glevel = 1;
    sp.dst = ua;
    sp.src_p = pitched_cell(g, sh.src_cell);
    sp.wavelet = sh.wavelet_dev;
    sp.ilevel = 1;
    CUDA_TRY(launch_sparse(sp, stor, s));
    void* prev = ua;  // u^{n-1}
    void* cur = ub;   // u^n
    for (int n = 1; n <= N; ++n) {
      StepArgs a = step_args(m, cur, prev);
      CUDA_TRY(run_step(m, a, s));
      std::swap(prev, cur);  // cur = u^{n+1}, prev = u^n
      if (n + 1 <= N) {
        sp.gsrc = cur;
        sp.glevel = n + 1;
        sp.dst = prev;
        sp.ilevel = n + 1;
        CUDA_TRY(launch_sparse(sp, stor, s));
      }
    }
    if (final_dev && si == nshots - 1) {
      CUDA_TRY(launch_pitched_to_dense(g, prev, final_dev, stor, s));
      CUDA_TRY(launch_pitched_to_dense(g, cur, final_dev + ncells, stor, s));
    }
  }
  return WAVE_OK;
}

// ---------------------------------------------------------------------------
// gradient (Algorithm 1)
// ---------------------------------------------------------------------------
struct GradWs {
  float* acc;
  float* comp;
  void* u0;
  void* u1;
  void* u2;  // second field pair (WAVE_SYMMETRIC_K: u^-; WAVE_EXACT_REVERSE: lambda), else null
  void* u3;
  float* resid;
  int64_t* recp;
  double* parts;
  double* scal;  // [0] k, [1] psi2, [2] e2, [3] C (no caller buffer), [4] sum grad^2, [6] C copy
};

static void carve_gradient(Carve& c, const wave_model_s* m, const wave_shot* shots, int32_t nshots, int mode,
                           GradWs* w) {
  int64_t maxres = 1;
  int32_t maxrec = 1;
  for (int s = 0; s < nshots; ++s) {
    maxres = std::max<int64_t>(maxres, (int64_t)(shots[s].nt + 1) * shots[s].nrec);
    maxrec = std::max(maxrec, shots[s].nrec);
  }
  const size_t eb = storage_bytes(m->d.storage);
  w->acc = c.take<float>(m->g.cells);
  w->comp = m->d.kahan ? c.take<float>(m->g.cells) : nullptr;
  w->u0 = c.take_bytes(m->g.cells * eb);
  w->u1 = c.take_bytes(m->g.cells * eb);
  const bool two = mode == WAVE_SYMMETRIC_K || mode == WAVE_EXACT_REVERSE;
  w->u2 = two ? c.take_bytes(m->g.cells * eb) : nullptr;
  w->u3 = two ? c.take_bytes(m->g.cells * eb) : nullptr;
  w->resid = c.take<float>(maxres);
  w->recp = c.take<int64_t>(maxrec);
  w->parts = c.take<double>(1024);
  w->scal = c.take<double>(8);
}

static wave_status validate_opts(const wave_model_s* m, const wave_gradient_opts* o) {
  if (!o) return WAVE_EINVAL;
  if (o->objective != WAVE_OBJ_L2 && o->objective != WAVE_OBJ_PATCH) return WAVE_EINVAL;
  if (o->mode < WAVE_SUPERPOSITION || o->mode > WAVE_EXACT_REVERSE) return WAVE_EINVAL;
  if (o->grad_wrt != WAVE_GRAD_MASS && o->grad_wrt != WAVE_GRAD_PARAM) return WAVE_EINVAL;
  if ((o->mode == WAVE_EXACT_STORED || o->mode == WAVE_EXACT_REVERSE) &&
      (o->batched || m->d.physics != WAVE_VELOCITY || m->d.storage != WAVE_F32))
    return WAVE_EUNSUPPORTED;
  if (o->mode == WAVE_SYMMETRIC_K && o->batched) return WAVE_EUNSUPPORTED;
  if (o->batched && !(m->d.ndim == 3 && m->d.physics == WAVE_VELOCITY && m->d.storage == WAVE_F32))
    return WAVE_EUNSUPPORTED;
  return WAVE_OK;
}

// Ratio r of the automatic k = r ||psi|| / ||f_adj|| (the stand-in for the
// calibration of Sec. 4.1: the smallest k at which FP32 still agrees with
// FP64).  Defaults: 1e-2 for Algorithm 1 in the velocity form; 5e-2 in the
// density form, whose FP32 cancellation in K(u^s,u^s) - K(u,u) is larger; 1
// for the +-k mean, which has no k^2 term to keep small.
static double default_ratio(const wave_model_s* m, const wave_gradient_opts* o) {
  if (o->k_ratio > 0.0) return o->k_ratio;
  if (o->mode == WAVE_SYMMETRIC_K) return 1.0;
  return m->d.physics == WAVE_DENSITY ? 5e-2 : 1e-2;
}

static double objective_weight(const wave_gradient_opts* o, const wave_shot& sh) {
  if (o->objective == WAVE_OBJ_L2) return 1.0;
  return sh.nrec > 0 ? 2.0 * o->patch_sign / sh.nrec : 0.0;
}

// Batched mode keeps every shot's two levels and residual traces resident.
struct BatchWs {
  float* acc;
  float* comp;
  std::vector<void*> u0, u1;
  std::vector<float*> resid;
  std::vector<int64_t*> recp;
  double* parts;
  double* scal;
};

static void carve_batched(Carve& c, const wave_model_s* m, const wave_shot* shots, int32_t nshots, BatchWs* w) {
  w->acc = c.take<float>(m->g.cells);
  w->comp = m->d.kahan ? c.take<float>(m->g.cells) : nullptr;
  w->u0.resize(nshots);
  w->u1.resize(nshots);
  w->resid.resize(nshots);
  w->recp.resize(nshots);
  for (int s = 0; s < nshots; ++s) {
    w->u0[s] = c.take<float>(m->g.cells);
    w->u1[s] = c.take<float>(m->g.cells);
    w->resid[s] = c.take<float>(std::max<int64_t>(1, (int64_t)(shots[s].nt + 1) * shots[s].nrec));
    w->recp[s] = c.take<int64_t>(std::max(1, shots[s].nrec));
  }
  w->parts = c.take<double>(1024);
  w->scal = c.take<double>(8);
}

// Exact mode: the forward history u^0..u^{N+1} of one shot at a time.
struct ExactWs {
  float* acc;
  float* hist;
  float* lam0;
  float* lam1;
  float* resid;
  int64_t* recp;
  double* parts;
  double* scal;
};

static void carve_exact(Carve& c, const wave_model_s* m, const wave_shot* shots, int32_t nshots, ExactWs* w) {
  int nmax = 1;
  int64_t maxres = 1;
  int32_t maxrec = 1;
  for (int s = 0; s < nshots; ++s) {
    nmax = std::max(nmax, shots[s].nt);
    maxres = std::max<int64_t>(maxres, (int64_t)(shots[s].nt + 1) * shots[s].nrec);
    maxrec = std::max(maxrec, shots[s].nrec);
  }
  w->acc = c.take<float>(m->g.cells);
  w->hist = c.take<float>((size_t)(nmax + 2) * m->g.cells);
  w->lam0 = c.take<float>(m->g.cells);
  w->lam1 = c.take<float>(m->g.cells);
  w->resid = c.take<float>(maxres);
  w->recp = c.take<int64_t>(maxrec);
  w->parts = c.take<double>(1024);
  w->scal = c.take<double>(8);
}

extern "C" wave_status wave_gradient_workspace_size(wave_model m, const wave_shot* shots, int32_t nshots,
                                                    const wave_gradient_opts* opts, size_t* bytes) {
  if (!m || !bytes) return WAVE_EINVAL;
  wave_status st = validate_shots(m, shots, nshots, false);
  if (st != WAVE_OK) return st;
  st = validate_opts(m, opts);
  if (st != WAVE_OK) return st;
  Carve c(nullptr);
  if (opts->mode == WAVE_EXACT_STORED) {
    ExactWs w;
    carve_exact(c, m, shots, nshots, &w);
  } else if (opts->batched) {
    BatchWs w;
    carve_batched(c, m, shots, nshots, &w);
  } else {
    GradWs w;
    carve_gradient(c, m, shots, nshots, opts->mode, &w);
  }
  *bytes = c.off;
  return WAVE_OK;
}


// Final scaling into grad_dev with the FP64 2-norm of the result (Sec. 4's
// K~, or the exact gradient), and the call's scalars for the metrics.
static wave_status finish_call(const wave_model_s* m, const float* acc, const double* kd, double inv_dt,
                               int superposition, bool chain_v, float* grad_dev, double* parts, double* scal,
                               const double* misfit_acc, double* grad_norm_dev, cudaStream_t s) {
  const Geom& g = m->g;
  CUDA_TRY(launch_finish(g, acc, kd, inv_dt, superposition, chain_v, m->param, grad_dev, parts, s));
  CUDA_TRY(launch_sum_final(parts, finish_parts(g.nx * g.ny * g.nz), 1.0, 0, scal + 4, s, grad_norm_dev));
  if (m->met.on) {
    CUDA_TRY(cudaMemcpyAsync(scal + 6, misfit_acc, sizeof(double), cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(mark(m, kEvAdjointEnd, s));
  }
  return WAVE_OK;
}

// Reset the metrics of the model for a new gradient call.
static cudaError_t metrics_begin(const wave_model_s* m, const wave_shot* shots, int32_t nshots, int mode,
                                 const double* scal) {
  auto& M = m->met;
  M.valid = M.on;
  if (!M.on) return cudaSuccess;
  M.used = 0;
  M.bytes = 0.0;
  M.launches = 0;
  M.units = 0.0;
  const double cells = (double)(m->g.nx * m->g.ny * m->g.nz);
  for (int i = 0; i < nshots; ++i) M.units += cells * shots[i].nt;
  M.scal = scal;
  M.mode = mode;
  return cudaSuccess;
}

// Standard adjoint over the stored forward history (Sec. 2.2 sensitivity
// analysis): forward with every level kept, then the adjoint recursion
// lambda^{j-1} = 2 lambda^j - lambda^{j+1} + dt^2/a (L lambda^j + f_adj^j) from
// lambda^{N+1} = lambda^N = 0, accumulating -(lambda^j - lambda^{j-1})(u^j - u^{j-1})
// (dt times the discrete Eq. kernel1).  The comparator of the superposition
// result; memory grows with N.
static wave_status gradient_exact(wave_model m, const wave_shot* shots, int32_t nshots,
                                  const wave_gradient_opts* opts, float* grad_dev, double* misfit_dev,
                                  double* k_dev, double* norm_dev, void* ws, cudaStream_t s) {
  const Geom& g = m->g;
  const double dt = m->d.dt;
  Carve c(ws);
  ExactWs w;
  carve_exact(c, m, shots, nshots, &w);
  double* kd = w.scal + 0;
  double* misfit_acc = misfit_dev ? misfit_dev : w.scal + 3;
  CUDA_TRY(cudaMemsetAsync(w.acc, 0, g.cells * sizeof(float), s));
  CUDA_TRY(cudaMemsetAsync(misfit_acc, 0, sizeof(double), s));
  CUDA_TRY(launch_set_k(kd, 1.0, s));  // the adjoint source enters unscaled
  CUDA_TRY(metrics_begin(m, shots, nshots, opts->mode, w.scal));
  auto level = [&](int n) { return w.hist + (size_t)n * g.cells; };
  for (int si = 0; si < nshots; ++si) {
    const wave_shot& sh = shots[si];
    const int N = sh.nt;
    const double wgt = objective_weight(opts, sh);
    CUDA_TRY(mark(m, kEvStart, s));
    CUDA_TRY(launch_pitch_indices(g, sh.rec_cells_dev, sh.nrec, w.recp, s));
    CUDA_TRY(cudaMemsetAsync(level(0), 0, 2 * g.cells * sizeof(float), s));
    SparseArgs gat = sparse_args(m, w.recp, sh.nrec);
    gat.observed = sh.observed_dev;
    gat.obs_ld = N + 1;
    gat.resid = w.resid;
    gat.gsrc = level(0);
    gat.glevel = 0;
    CUDA_TRY(launch_sparse(gat, WAVE_F32, s));
    gat.gsrc = level(1);
    gat.glevel = 1;
    CUDA_TRY(launch_sparse(gat, WAVE_F32, s));
    // The step takes the same operations as wave_forward and the other modes
    // (f^n subtracted from the level the step overwrites, then the in-place
    // update), so the stored levels, traces and misfit are bitwise those of
    // the forward: u^{n-1} is copied into the slot of u^{n+1} first.
    SparseArgs inj = sparse_args(m, w.recp, 0);
    inj.src_p = pitched_cell(g, sh.src_cell);
    inj.wavelet = sh.wavelet_dev;
    for (int n = 1; n <= N; ++n) {
      CUDA_TRY(cudaMemcpyAsync(level(n + 1), level(n - 1), g.cells * sizeof(float), cudaMemcpyDeviceToDevice, s));
      inj.dst = level(n + 1);
      inj.ilevel = n;
      CUDA_TRY(launch_sparse(inj, WAVE_F32, s));
      StepArgs a = step_args(m, level(n), level(n + 1));
      CUDA_TRY(run_step(m, a, s));
      if (n + 1 <= N) {
        gat.gsrc = level(n + 1);
        gat.glevel = n + 1;
        CUDA_TRY(launch_sparse(gat, WAVE_F32, s));
      }
    }
    const int64_t nres = (int64_t)(N + 1) * sh.nrec;
    if (nres > 0) {
      const int np = reduce_parts(nres);
      CUDA_TRY(launch_sumsq_partial(w.resid, nullptr, nres, w.parts, np, s));
      CUDA_TRY(launch_sum_final(w.parts, np, 0.5 * wgt * dt, 1, misfit_acc, s));
    }
    CUDA_TRY(mark(m, kEvForwardEnd, s));
    // adjoint: lambda^{N+1} = lambda^N = 0
    CUDA_TRY(cudaMemsetAsync(w.lam0, 0, g.cells * sizeof(float), s));
    CUDA_TRY(cudaMemsetAsync(w.lam1, 0, g.cells * sizeof(float), s));
    float* lam_next = w.lam0;  // lambda^{j+1}
    float* lam_cur = w.lam1;   // lambda^j
    SparseArgs adj = sparse_args(m, w.recp, sh.nrec);
    adj.resid_in = w.resid;
    adj.k_dev = kd;
    adj.weight = (float)wgt;
    for (int j = N; j >= 1; --j) {
      adj.dst = lam_next;
      adj.ilevel = j;
      CUDA_TRY(launch_sparse(adj, WAVE_F32, s));
      StepArgs a = step_args(m, lam_cur, lam_next);
      a.acc = w.acc;
      a.acc_scale = -1.f;
      a.acc_mass = 1;
      a.mix_a = level(j);
      a.mix_b = level(j - 1);
      CUDA_TRY(run_step(m, a, s));
      std::swap(lam_cur, lam_next);  // lam_cur = lambda^{j-1}
    }
    if (si + 1 < nshots) CUDA_TRY(mark(m, kEvAdjointEnd, s));
  }
  CUDA_TRY(cudaMemsetAsync(kd, 0, sizeof(double), s));   // no k in this mode
  wave_status st = finish_call(m, w.acc, kd, 1.0 / dt, 0, opts->grad_wrt == WAVE_GRAD_PARAM, grad_dev, w.parts,
                               w.scal, misfit_acc, norm_dev, s);
  if (st != WAVE_OK) return st;
  if (k_dev) CUDA_TRY(cudaMemsetAsync(k_dev, 0, sizeof(double), s));
  return WAVE_OK;
}

static wave_status gradient_batched(wave_model m, const wave_shot* shots, int32_t nshots,
                                    const wave_gradient_opts* opts, float* grad_dev, double* misfit_dev,
                                    double* k_dev, double* norm_dev, void* ws, cudaStream_t s) {
  const Geom& g = m->g;
  const double dt = m->d.dt;
  Carve c(ws);
  BatchWs w;
  carve_batched(c, m, shots, nshots, &w);
  double* kd = w.scal + 0;
  double* misfit_acc = misfit_dev ? misfit_dev : w.scal + 3;
  CUDA_TRY(metrics_begin(m, shots, nshots, opts->mode, w.scal));
  CUDA_TRY(mark(m, kEvStart, s));
  CUDA_TRY(cudaMemsetAsync(w.acc, 0, g.cells * sizeof(float), s));
  if (w.comp) CUDA_TRY(cudaMemsetAsync(w.comp, 0, g.cells * sizeof(float), s));
  CUDA_TRY(cudaMemsetAsync(misfit_acc, 0, sizeof(double), s));
  const bool auto_k = !(opts->k > 0.0);
  if (!auto_k) CUDA_TRY(launch_set_k(kd, opts->k, s));
  const double ratio = default_ratio(m, opts);
  std::vector<void*> prev(nshots), cur(nshots);
  std::vector<SparseArgs> sp(nshots);
  int nmax = 0;
  for (int si = 0; si < nshots; ++si) {
    const wave_shot& sh = shots[si];
    nmax = std::max(nmax, sh.nt);
    CUDA_TRY(launch_pitch_indices(g, sh.rec_cells_dev, sh.nrec, w.recp[si], s));
    CUDA_TRY(cudaMemsetAsync(w.u0[si], 0, g.cells * sizeof(float), s));
    CUDA_TRY(cudaMemsetAsync(w.u1[si], 0, g.cells * sizeof(float), s));
    SparseArgs a = sparse_args(m, w.recp[si], sh.nrec);
    a.observed = sh.observed_dev;
    a.obs_ld = sh.nt + 1;
    a.resid = w.resid[si];
    a.gsrc = w.u0[si];
    a.glevel = 0;
    CUDA_TRY(launch_sparse(a, WAVE_F32, s));
    a.gsrc = w.u1[si];
    a.glevel = 1;
    a.dst = w.u0[si];
    a.src_p = pitched_cell(g, sh.src_cell);
    a.wavelet = sh.wavelet_dev;
    a.ilevel = 1;
    CUDA_TRY(launch_sparse(a, WAVE_F32, s));
    sp[si] = a;
    prev[si] = w.u0[si];
    cur[si] = w.u1[si];
  }
  StepArgs base = step_args(m, nullptr, nullptr);
  base.acc = w.acc;
  base.comp = w.comp;
  // ---- forward: all shots start at t = 0 --------------------------------
  for (int n = 1; n <= nmax; ++n) {
    BatchArgs b;
    memset(&b, 0, sizeof(b));
    b.base = base;
    b.base.acc_scale = 1.f;
    b.err = m->err;
    b.wait_limit_cycles = m->wait_limit_cycles;
    b.debug_stall = m->debug_stall;
    for (int si = 0; si < nshots; ++si) {
      if (shots[si].nt < n) continue;
      b.cur[b.nshots] = static_cast<const float*>(cur[si]);
      b.prev[b.nshots] = static_cast<float*>(prev[si]);
      b.accf[b.nshots] = n <= shots[si].nt - 1;
      if (++b.nshots == kMaxBatch) {
        CUDA_TRY(run_batched(m, b, s));
        b.nshots = 0;
      }
    }
    if (b.nshots) CUDA_TRY(run_batched(m, b, s));
    for (int si = 0; si < nshots; ++si) {
      if (shots[si].nt < n) continue;
      std::swap(prev[si], cur[si]);
      if (n + 1 <= shots[si].nt) {
        sp[si].gsrc = cur[si];
        sp[si].glevel = n + 1;
        sp[si].dst = prev[si];
        sp[si].ilevel = n + 1;
        CUDA_TRY(launch_sparse(sp[si], WAVE_F32, s));
      }
    }
  }
  // ---- cost and k -----------------------------------------------------------
  for (int si = 0; si < nshots; ++si) {
    const wave_shot& sh = shots[si];
    const double wgt = objective_weight(opts, sh);
    const int64_t nres = (int64_t)(sh.nt + 1) * sh.nrec;
    if (nres > 0) {
      const int np = reduce_parts(nres);
      CUDA_TRY(launch_sumsq_partial(w.resid[si], nullptr, nres, w.parts, np, s));
      CUDA_TRY(launch_sum_final(w.parts, np, 0.5 * wgt * dt, 1, misfit_acc, s));
    }
  }
  if (auto_k) {
    const wave_shot& sh = shots[0];
    const int N = sh.nt;
    const int np1 = reduce_parts(N);
    CUDA_TRY(launch_sumsq_partial(sh.wavelet_dev + 1, nullptr, N, w.parts, np1, s));
    CUDA_TRY(launch_sum_final(w.parts, np1, 1.0, 0, w.scal + 1, s));
    const int64_t ne = (int64_t)N * sh.nrec;
    if (ne > 0) {
      const int np2 = reduce_parts(ne);
      CUDA_TRY(launch_sumsq_partial(w.resid[0] + sh.nrec, nullptr, ne, w.parts, np2, s));
      CUDA_TRY(launch_sum_final(w.parts, np2, 1.0, 0, w.scal + 2, s));
    } else {
      CUDA_TRY(cudaMemsetAsync(w.scal + 2, 0, sizeof(double), s));
    }
    CUDA_TRY(launch_auto_k(w.scal + 1, w.scal + 2, ratio, objective_weight(opts, sh), kd, s));
  }
  CUDA_TRY(mark(m, kEvForwardEnd, s));
  // ---- superposed pass: shot s runs j = N_s..1 at global steps t = j --------
  std::vector<void*> us_cur(nshots), us_next(nshots);
  std::vector<SparseArgs> sb(nshots);
  for (int si = 0; si < nshots; ++si) {
    us_cur[si] = prev[si];   // u^{N}
    us_next[si] = cur[si];   // u^{N+1}
    sb[si] = sparse_args(m, w.recp[si], shots[si].nrec);
    sb[si].src_p = pitched_cell(g, shots[si].src_cell);
    sb[si].wavelet = shots[si].wavelet_dev;
    sb[si].resid_in = w.resid[si];
    sb[si].k_dev = kd;
    sb[si].weight = (float)objective_weight(opts, shots[si]);
  }
  for (int t = nmax; t >= 1; --t) {
    for (int si = 0; si < nshots; ++si) {
      if (shots[si].nt < t) continue;
      sb[si].dst = us_next[si];
      sb[si].ilevel = t;
      CUDA_TRY(launch_sparse(sb[si], WAVE_F32, s));
    }
    BatchArgs b;
    memset(&b, 0, sizeof(b));
    b.base = base;
    b.base.acc_scale = -1.f;
    b.err = m->err;
    b.wait_limit_cycles = m->wait_limit_cycles;
    b.debug_stall = m->debug_stall;
    for (int si = 0; si < nshots; ++si) {
      if (shots[si].nt < t) continue;
      b.cur[b.nshots] = static_cast<const float*>(us_cur[si]);
      b.prev[b.nshots] = static_cast<float*>(us_next[si]);
      b.accf[b.nshots] = 1;
      if (++b.nshots == kMaxBatch) {
        CUDA_TRY(run_batched(m, b, s));
        b.nshots = 0;
      }
    }
    if (b.nshots) CUDA_TRY(run_batched(m, b, s));
    for (int si = 0; si < nshots; ++si) {
      if (shots[si].nt < t) continue;
      std::swap(us_cur[si], us_next[si]);
    }
  }
  wave_status st = finish_call(m, w.acc, kd, 1.0 / dt, 1, opts->grad_wrt == WAVE_GRAD_PARAM, grad_dev, w.parts,
                               w.scal, misfit_acc, norm_dev, s);
  if (st != WAVE_OK) return st;
  if (k_dev) CUDA_TRY(cudaMemcpyAsync(k_dev, kd, sizeof(double), cudaMemcpyDeviceToDevice, s));
  return WAVE_OK;
}


extern "C" wave_status wave_adjoint_sensitivity(wave_model m, const wave_shot* shots, int32_t nshots,
                                                const wave_gradient_opts* opts, float* grad_dev,
                                                double* misfit_dev, double* k_dev, double* grad_norm_dev,
                                                void* ws, size_t ws_bytes, void* stream) {
  if (!m || !grad_dev) return WAVE_EINVAL;
  wave_status st = validate_shots(m, shots, nshots, false);
  if (st != WAVE_OK) return st;
  st = validate_opts(m, opts);
  if (st != WAVE_OK) return st;
  if (opts->objective == WAVE_OBJ_PATCH && !(opts->patch_sign == 1.0 || opts->patch_sign == -1.0)) return WAVE_EINVAL;
  size_t need = 0;
  wave_gradient_workspace_size(m, shots, nshots, opts, &need);
  if (!ws || ws_bytes < need || reinterpret_cast<uintptr_t>(ws) % 256) return WAVE_EWORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  if (opts->mode == WAVE_EXACT_STORED)
    return gradient_exact(m, shots, nshots, opts, grad_dev, misfit_dev, k_dev, grad_norm_dev, ws, s);
  if (opts->batched) return gradient_batched(m, shots, nshots, opts, grad_dev, misfit_dev, k_dev, grad_norm_dev, ws, s);
  const Geom& g = m->g;
  const int stor = m->d.storage;
  const size_t eb = storage_bytes(stor);
  const double dt = m->d.dt;
  Carve c(ws);
  GradWs w;
  carve_gradient(c, m, shots, nshots, opts->mode, &w);
  double* kd = w.scal + 0;
  double* misfit_acc = misfit_dev ? misfit_dev : w.scal + 3;
  const bool sym = opts->mode == WAVE_SYMMETRIC_K;
  const bool rev = opts->mode == WAVE_EXACT_REVERSE;
  CUDA_TRY(metrics_begin(m, shots, nshots, opts->mode, w.scal));

  CUDA_TRY(cudaMemsetAsync(w.acc, 0, g.cells * sizeof(float), s));
  if (w.comp) CUDA_TRY(cudaMemsetAsync(w.comp, 0, g.cells * sizeof(float), s));
  CUDA_TRY(cudaMemsetAsync(misfit_acc, 0, sizeof(double), s));
  const bool auto_k = !rev && !(opts->k > 0.0);
  if (rev) CUDA_TRY(launch_set_k(kd, 1.0, s));  // the adjoint source enters unscaled
  else if (!auto_k) CUDA_TRY(launch_set_k(kd, opts->k, s));
  const double ratio = default_ratio(m, opts);
  // both fields of WAVE_SYMMETRIC_K advance in one launch where the batched kernel applies
  const bool fuse2 = sym && m->d.ndim == 3 && m->d.physics == WAVE_VELOCITY && stor == WAVE_F32;

  for (int si = 0; si < nshots; ++si) {
    const wave_shot& sh = shots[si];
    const int N = sh.nt;
    const double wgt = objective_weight(opts, sh);
    if (si > 0) CUDA_TRY(mark(m, kEvAdjointEnd, s));
    CUDA_TRY(mark(m, kEvStart, s));
    CUDA_TRY(launch_pitch_indices(g, sh.rec_cells_dev, sh.nrec, w.recp, s));
    CUDA_TRY(cudaMemsetAsync(w.u0, 0, g.cells * eb, s));
    CUDA_TRY(cudaMemsetAsync(w.u1, 0, g.cells * eb, s));
    // levels 0 and 1 (Eq. IC), then inject f^1 into u^0
    SparseArgs sp = sparse_args(m, w.recp, sh.nrec);
    sp.observed = sh.observed_dev;
    sp.obs_ld = N + 1;
    sp.resid = w.resid;
    sp.gsrc = w.u0;
    sp.glevel = 0;
    CUDA_TRY(launch_sparse(sp, stor, s));
    sp.gsrc = w.u1;
    sp.glevel = 1;
    sp.dst = w.u0;
    sp.src_p = pitched_cell(g, sh.src_cell);
    sp.wavelet = sh.wavelet_dev;
    sp.ilevel = 1;
    CUDA_TRY(launch_sparse(sp, stor, s));
    // ---- forward: propagate, adjoint source, -K(u,u) ------------------
    void* prev = w.u0;
    void* cur = w.u1;
    for (int n = 1; n <= N; ++n) {
      StepArgs a = step_args(m, cur, prev);
      a.acc = w.acc;
      a.comp = w.comp;
      a.acc_scale = 1.f;
      a.acc_mass = !(sym || rev) && n <= N - 1;   // the two-field modes need no K(u,u)
      a.acc_stiff = !(sym || rev) && n <= N - 1;
      CUDA_TRY(run_step(m, a, s));
      std::swap(prev, cur);  // cur = u^{n+1}
      if (n + 1 <= N) {
        sp.gsrc = cur;
        sp.glevel = n + 1;
        sp.dst = prev;
        sp.ilevel = n + 1;
        CUDA_TRY(launch_sparse(sp, stor, s));
      }
    }
    // ---- cost (Eq. cost1 / cost2) and k -------------------------------
    const int64_t nres = (int64_t)(N + 1) * sh.nrec;
    if (nres > 0) {
      const int np = reduce_parts(nres);
      CUDA_TRY(launch_sumsq_partial(w.resid, nullptr, nres, w.parts, np, s));
      CUDA_TRY(launch_sum_final(w.parts, np, 0.5 * wgt * dt, 1, misfit_acc, s));
    }
    if (si == 0 && auto_k) {
      const int np1 = reduce_parts(N);
      CUDA_TRY(launch_sumsq_partial(sh.wavelet_dev + 1, nullptr, N, w.parts, np1, s));
      CUDA_TRY(launch_sum_final(w.parts, np1, 1.0, 0, w.scal + 1, s));
      const int64_t ne = (int64_t)N * sh.nrec;
      if (ne > 0) {
        const int np2 = reduce_parts(ne);
        CUDA_TRY(launch_sumsq_partial(w.resid + sh.nrec, nullptr, ne, w.parts, np2, s));
        CUDA_TRY(launch_sum_final(w.parts, np2, 1.0, 0, w.scal + 2, s));
      } else {
        CUDA_TRY(cudaMemsetAsync(w.scal + 2, 0, sizeof(double), s));
      }
      CUDA_TRY(launch_auto_k(w.scal + 1, w.scal + 2, ratio, wgt, kd, s));
    }
    CUDA_TRY(mark(m, kEvForwardEnd, s));
    // prev holds u^N, cur holds u^{N+1}
    if (rev) {
      // ---- u backward by time reversal beside lambda (Eq. kernel1 mixed term)
      CUDA_TRY(cudaMemsetAsync(w.u2, 0, g.cells * eb, s));
      CUDA_TRY(cudaMemsetAsync(w.u3, 0, g.cells * eb, s));
      void* u_c = prev;   // u^j
      void* u_n = cur;    // u^{j+1}, overwritten with u^{j-1}
      void* l_c = w.u3;   // lambda^j
      void* l_n = w.u2;   // lambda^{j+1}, overwritten with lambda^{j-1}
      SparseArgs fs = sparse_args(m, w.recp, 0);
      fs.src_p = pitched_cell(g, sh.src_cell);
      fs.wavelet = sh.wavelet_dev;
      SparseArgs adj = sparse_args(m, w.recp, sh.nrec);
      adj.resid_in = w.resid;
      adj.k_dev = kd;
      adj.weight = (float)wgt;
      // 3D: u and lambda advance in one launch, the mixed term taken from registers
      const bool fused = m->d.ndim == 3 && g.plane < ((int64_t)1 << 31);
      for (int j = N; j >= 1; --j) {
        fs.dst = u_n;
        fs.ilevel = j;
        CUDA_TRY(launch_sparse(fs, stor, s));
        adj.dst = l_n;
        adj.ilevel = j;
        CUDA_TRY(launch_sparse(adj, stor, s));
        if (fused) {
          BatchArgs b;
          memset(&b, 0, sizeof(b));
          b.base = step_args(m, nullptr, nullptr);
          b.base.acc = w.acc;
          b.base.acc_scale = -1.f;
          b.err = m->err;
          b.wait_limit_cycles = m->wait_limit_cycles;
          b.debug_stall = m->debug_stall;
          b.nshots = 2;
          b.cur[0] = static_cast<const float*>(u_c);
          b.prev[0] = static_cast<float*>(u_n);
          b.cur[1] = static_cast<const float*>(l_c);
          b.prev[1] = static_cast<float*>(l_n);
          b.accf[0] = 0.f;
          b.accf[1] = 1.f;
          b.pair_mix = 1;
          CUDA_TRY(run_batched(m, b, s));
          std::swap(u_c, u_n);
          std::swap(l_c, l_n);
          continue;
        }
        CUDA_TRY(run_step(m, step_args(m, u_c, u_n), s));
        StepArgs a = step_args(m, l_c, l_n);
        a.acc = w.acc;
        a.acc_scale = -1.f;
        a.acc_mass = 1;
        a.mix_a = static_cast<const float*>(u_c);
        a.mix_b = static_cast<const float*>(u_n);
        CUDA_TRY(run_step(m, a, s));
        std::swap(u_c, u_n);
        std::swap(l_c, l_n);
      }
      continue;
    }
    if (sym) {
      // ---- u^+ (k) on (prev, cur), u^- (-k) on copies of them ---------
      CUDA_TRY(cudaMemcpyAsync(w.u2, prev, g.cells * eb, cudaMemcpyDeviceToDevice, s));
      CUDA_TRY(cudaMemcpyAsync(w.u3, cur, g.cells * eb, cudaMemcpyDeviceToDevice, s));
      void* fc[2] = {prev, w.u2};   // u^{+-,j}
      void* fn[2] = {cur, w.u3};    // u^{+-,j+1}, overwritten with u^{+-,j-1}
      SparseArgs sf[2];
      for (int f = 0; f < 2; ++f) {
        sf[f] = sparse_args(m, w.recp, sh.nrec);
        sf[f].src_p = pitched_cell(g, sh.src_cell);
        sf[f].wavelet = sh.wavelet_dev;
        sf[f].resid_in = w.resid;
        sf[f].k_dev = kd;
        sf[f].weight = (float)(f == 0 ? wgt : -wgt);   // force f +- k f_adj
      }
      for (int j = N; j >= 1; --j) {
        for (int f = 0; f < 2; ++f) {
          sf[f].dst = fn[f];
          sf[f].ilevel = j;
          CUDA_TRY(launch_sparse(sf[f], stor, s));
        }
        if (fuse2) {
          BatchArgs b;
          memset(&b, 0, sizeof(b));
          b.base = step_args(m, nullptr, nullptr);
          b.base.acc = w.acc;
          b.base.comp = w.comp;
          b.base.acc_scale = -1.f;
          b.err = m->err;
          b.wait_limit_cycles = m->wait_limit_cycles;
          b.debug_stall = m->debug_stall;
          b.nshots = 2;
          for (int f = 0; f < 2; ++f) {
            b.cur[f] = static_cast<const float*>(fc[f]);
            b.prev[f] = static_cast<float*>(fn[f]);
            b.accf[f] = f == 0 ? 1.f : -1.f;   // -K(u^+,u^+) ... +K(u^-,u^-)
          }
          CUDA_TRY(run_batched(m, b, s));
        } else {
          for (int f = 0; f < 2; ++f) {
            StepArgs a = step_args(m, fc[f], fn[f]);
            a.acc = w.acc;
            a.comp = w.comp;
            a.acc_scale = f == 0 ? -1.f : 1.f;
            a.acc_mass = 1;
            a.acc_stiff = j <= N - 1;
            CUDA_TRY(run_step(m, a, s));
          }
        }
        for (int f = 0; f < 2; ++f) std::swap(fc[f], fn[f]);
      }
      continue;
    }
    // ---- superposed pass: u^s from (u^{N+1}, u^N), +K(u^s,u^s) ----------
    void* us_cur = prev;   // u^{s,j}
    void* us_next = cur;   // u^{s,j+1}, overwritten with u^{s,j-1}
    SparseArgs sb = sparse_args(m, w.recp, sh.nrec);
    sb.src_p = pitched_cell(g, sh.src_cell);
    sb.wavelet = sh.wavelet_dev;
    sb.resid_in = w.resid;
    sb.k_dev = kd;
    sb.weight = (float)wgt;
    for (int j = N; j >= 1; --j) {
      sb.dst = us_next;
      sb.ilevel = j;
      CUDA_TRY(launch_sparse(sb, stor, s));
      StepArgs a = step_args(m, us_cur, us_next);
      a.acc = w.acc;
      a.comp = w.comp;
      a.acc_scale = -1.f;
      a.acc_mass = 1;
      a.acc_stiff = j <= N - 1;
      CUDA_TRY(run_step(m, a, s));
      std::swap(us_cur, us_next);  // us_cur = u^{s,j-1}, us_next = u^{s,j}
    }
  }
  // ---- K~ = (K(u^s,u^s) - K(u,u)) / 2k (Eq. superposedkernel); the
  // symmetric pair divides by 4k, the reverse-time mode by nothing ----------
  const bool chain_v = opts->grad_wrt == WAVE_GRAD_PARAM && m->d.physics == WAVE_VELOCITY;
  if (rev) CUDA_TRY(cudaMemsetAsync(kd, 0, sizeof(double), s));   // no k in this mode
  wave_status fst = finish_call(m, w.acc, kd, (sym ? 0.5 : 1.0) / dt, rev ? 0 : 1, chain_v, grad_dev, w.parts,
                                w.scal, misfit_acc, grad_norm_dev, s);
  if (fst != WAVE_OK) return fst;
  if (k_dev && rev) CUDA_TRY(cudaMemsetAsync(k_dev, 0, sizeof(double), s));
  else if (k_dev) CUDA_TRY(cudaMemcpyAsync(k_dev, kd, sizeof(double), cudaMemcpyDeviceToDevice, s));
  return WAVE_OK;
}

// ---------------------------------------------------------------------------
// per-call metrics
// ---------------------------------------------------------------------------
extern "C" wave_status wave_model_set_metrics(wave_model m, int32_t on) {
  if (!m) return WAVE_EINVAL;
  m->met.on = on != 0;
  m->met.valid = false;
  return WAVE_OK;
}

extern "C" wave_status wave_gradient_metrics_read(wave_model m, wave_gradient_metrics* out) {
  if (!m || !out) return WAVE_EINVAL;
  auto& M = m->met;
  if (!M.on || !M.valid || M.used == 0 || !M.scal) return WAVE_EINVAL;
  CUDA_TRY(cudaEventSynchronize(M.ev[M.used - 1]));
  double sc[8];
  CUDA_TRY(cudaMemcpy(sc, M.scal, sizeof(sc), cudaMemcpyDeviceToHost));
  memset(out, 0, sizeof(*out));
  out->misfit = sc[6];
  out->k = sc[0];
  out->grad_l2 = sqrt(sc[4]);
  double fwd = 0.0, adj = 0.0;
  for (size_t i = 1; i < M.used; ++i) {
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, M.ev[i - 1], M.ev[i]));
    if (M.kind[i] == kEvForwardEnd) fwd += ms;
    else if (M.kind[i] == kEvAdjointEnd) adj += ms;
  }
  float total = 0.f;
  CUDA_TRY(cudaEventElapsedTime(&total, M.ev[0], M.ev[M.used - 1]));
  out->forward_ms = fwd;
  out->adjoint_ms = adj;
  out->total_ms = total;
  out->step_bytes = M.bytes;
  out->cell_updates = M.units;
  out->step_launches = (int64_t)M.launches;
  // the optional end-of-call check for non-finite results
  if (!isfinite(out->misfit) || !isfinite(out->grad_l2) || !isfinite(out->k)) return WAVE_ENONFINITE;
  return WAVE_OK;
}

// ---------------------------------------------------------------------------
// misfit
// ---------------------------------------------------------------------------
extern "C" size_t wave_misfit_scratch_size(int64_t count) {
  return (size_t)reduce_parts(count < 1 ? 1 : count) * sizeof(double);
}

extern "C" wave_status misfit(const float* syn_dev, const float* obs_dev, int64_t count, double dt, double weight,
                              double* out_dev, void* scratch_dev, size_t scratch_bytes, void* stream) {
  if (!out_dev || count < 0 || !(dt > 0)) return WAVE_EINVAL;
  if (count > 0 && !syn_dev) return WAVE_EINVAL;
  const int np = reduce_parts(count < 1 ? 1 : count);
  if (!scratch_dev || scratch_bytes < (size_t)np * sizeof(double) ||
      reinterpret_cast<uintptr_t>(scratch_dev) % 8)
    return WAVE_EWORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  double* parts = static_cast<double*>(scratch_dev);
  CUDA_TRY(launch_sumsq_partial(syn_dev, obs_dev, count, parts, np, s));
  CUDA_TRY(launch_sum_final(parts, np, 0.5 * weight * dt, 0, out_dev, s));
  return WAVE_OK;
}
