// C-ABI layer of libwcns: argument validation, context scratch, stream ordering,
// CUDA-graph replay of RK3 steps, sticky device status.  See include/wcns.h.
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/wcns.h"
#include "wcns_grid_check.h"
#include "wcns_internal.h"

using namespace wcns;

struct wcns_ctx {
  wcns_grid g;
  wcns_params p;
  Scheme s;
  GridInfo gi;
  Faces<double> faces;   // boundary faces (active == 0: the grid's bc only)
  cudaStream_t stream;
  int device;
  size_t elem;           // element size in bytes
  size_t nelem;          // elements of one grid buffer (nvar * ny * pitch)
  void* u1;              // stage states
  void* u2;
  void* u3;              // third stage state (RK4 only)
  void* R;               // L_x planes (2D)
  void* host_state;      // device copy used by wcns_step_host (lazy)
  void* ring;            // partial-stage ring of the banded 2D stage (lazy, wcns_set_stage_form)
  bool banded;           // stages run banded (wcns_set_stage_form)
  unsigned* d_band;      // banded stage counters (kBandCounterWords, in scal)
  void* adj1;            // adjoint stage cotangents (lazy)
  void* adj2;
  // small device scalars (one allocation)
  void* scal;
  StepDt* d_dt;
  double* d_t;
  long long* d_steps;
  int* d_err;
  unsigned long long* d_fallbacks;
  unsigned int* d_counters;   // [8]
  unsigned long long* d_wave; // fused CFL maxima slots of a step's last stage (2D Euler), 2 * kWaveSlots
  double* d_out;              // [8]
  double* d_partials;         // [kMaxRedBlocks * 2]
  // 2D Euler: each step's last stage reduces the next step's CFL maxima (fused epilogue)
  bool fuse_wave;
  // graphs of one RK step: graph starts with the CFL kernel, graph_next with the step
  // record from the maxima of the previous step
  cudaGraphExec_t graph;
  cudaGraphExec_t graph_next;
  const void* graph_u;
  double graph_dt, graph_tend;
  // per-kernel event timing (benchmarks)
  bool prof_on;
  struct ProfEvent { int kind; cudaEvent_t a, b; };
  std::vector<ProfEvent> prof;
  size_t prof_used;
};

namespace {
enum ProfKind { kProfSweepXRhs = 0, kProfSweepYRhs, kProfSweepXStage1D, kProfSweepXLx, kProfSweepYStage, kProfDt,
                kProfReduce, kProfAdjX, kProfAdjY, kProfDtFused, kProfStageBand, kProfCount };
const char* const kProfNames[kProfCount] = {"sweep_x_rhs", "sweep_y_rhs", "sweep_x_stage_1d", "sweep_x_lx_2d",
                                            "sweep_y_stage_2d", "dt_cfl", "reduce", "adjoint_x", "adjoint_y", "dt_from_maxima",
                                            "stage_band_2d"};
}  // namespace

namespace {

wcns_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return WCNS_OK;
  if (e == cudaErrorMemoryAllocation) return WCNS_ERR_NOMEM;
  return WCNS_ERR_CUDA;
}

#define WCNS_TRY(expr)                               \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) return from_cuda(e_);     \
  } while (0)

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }


wcns_status check_params(const wcns_params* p, int dtype, int nvar, int ndim) {
  if (p->system != WCNS_ADVECTION && p->system != WCNS_EULER) return WCNS_ERR_ARG;
  if (p->weights < WCNS_W_JS || p->weights > WCNS_W_M) return WCNS_ERR_ARG;
  if (p->flux < WCNS_FLUX_LLF || p->flux > WCNS_FLUX_LLF_FROZEN) return WCNS_ERR_ARG;
  if (p->z_p != 1 && p->z_p != 2) return WCNS_ERR_ARG;
  if (p->integrator != WCNS_RK3 && p->integrator != WCNS_RK4) return WCNS_ERR_ARG;
  if (p->family != WCNS_FAMILY_WCNS && p->family != WCNS_FAMILY_WENO) return WCNS_ERR_ARG;
  if (!(p->eps > 0.0) || !(p->gamma > 1.0) || !(p->cfl > 0.0) || !(p->xi > 0.0)) return WCNS_ERR_ARG;
  if (!(p->kappa > 0.0) || p->cv < 0.0) return WCNS_ERR_ARG;
  // in single precision eps^2 must stay a normal number for the JS and M weights
  if (dtype == WCNS_F32 && (p->weights == WCNS_W_JS || p->weights == WCNS_W_M) && p->eps < 1e-18)
    return WCNS_ERR_ARG;
  if (p->system == WCNS_ADVECTION && nvar != 1) return WCNS_ERR_UNSUPPORTED;
  if (p->system == WCNS_EULER && !((ndim == 1 && nvar == 3) || (ndim == 2 && nvar == 4)))
    return WCNS_ERR_UNSUPPORTED;
  if (p->flux == WCNS_FLUX_LLF_FROZEN && (!(p->alpha[0] >= 0.0) || !(p->alpha[1] >= 0.0))) return WCNS_ERR_ARG;
  return WCNS_OK;
}

Scheme make_scheme(const wcns_params* p) {
  Scheme s{};
  s.system = p->system;
  s.weights = p->weights;
  s.flux = p->flux;
  s.characteristic = p->characteristic ? 1 : 0;
  s.zp = p->z_p;
  s.renorm = p->renorm ? 1 : 0;
  s.gamma = p->gamma;
  s.eps = p->eps;
  s.xi = p->xi;
  s.cv = p->cv;
  s.harten = p->harten;
  for (int d = 0; d < 2; ++d)
    s.speed[d] = (p->system == WCNS_ADVECTION) ? p->adv_speed[d] : p->alpha[d];
  fill_family_tables(s, p->family, p->kappa);
  return s;
}

template <typename F64, typename F32>
cudaError_t by_type(int dtype, F64 f64, F32 f32) {
  return dtype == WCNS_F64 ? f64() : f32();
}

bool by_type_bool(int dtype, bool f64, bool f32) { return dtype == WCNS_F64 ? f64 : f32; }

// The banded stage's counters sit in the context's scalar block at byte 1024.
static_assert(1024 + sizeof(unsigned) * kBandCounterWords <= 4096, "band counters fit the scalar block");

// Runs `f` (one kernel launch), bracketed by events when per-kernel timing is on.
template <class F>
cudaError_t timed(wcns_ctx* c, int kind, F f) {
  if (!c->prof_on) return f();
  if (c->prof_used == c->prof.size()) {
    wcns_ctx::ProfEvent ev{};
    if (cudaEventCreate(&ev.a) != cudaSuccess || cudaEventCreate(&ev.b) != cudaSuccess) return cudaErrorMemoryAllocation;
    c->prof.push_back(ev);
  }
  wcns_ctx::ProfEvent& ev = c->prof[c->prof_used++];
  ev.kind = kind;
  cudaError_t e = cudaEventRecord(ev.a, c->stream);
  if (e != cudaSuccess) return e;
  if ((e = f()) != cudaSuccess) return e;
  return cudaEventRecord(ev.b, c->stream);
}

// Stage coefficients: TVD-RK3 form out = a*un + b*(u + dt*L), or (general) the form
// out = a*un + b*u + e*dt*L + c1*X1 + c2*X2.
struct StageCoef {
  double a, b;
  bool general;
  double e, c1, c2;
  const void* X1;
  const void* X2;
  double cstage;  // the state the stage evaluates L on is at t0 + cstage * dt
  bool last;      // the stage completes an RK step (fused CFL maxima of its output)
};

template <typename T>
cudaError_t sweeps(wcns_ctx* c, const void* u, const void* un, void* out, bool stage_mode, const StageCoef& k) {
  SweepCall<T> x{};
  x.u = static_cast<const T*>(u);
  x.fallbacks = c->d_fallbacks;
  x.general = k.general;
  x.e = k.e; x.c1 = k.c1; x.c2 = k.c2;
  x.X1 = static_cast<const T*>(k.X1);
  x.X2 = static_cast<const T*>(k.X2);
  x.faces = &c->faces;
  x.cstage = k.cstage;
  x.tnow = c->d_t;
  x.status = c->d_err;
  if (c->g.ndim == 1) {
    x.un = static_cast<const T*>(un);
    x.out = static_cast<T*>(out);
    x.dt = stage_mode ? c->d_dt : nullptr;
    x.a = k.a; x.b = k.b;
    x.stage = stage_mode;
    return timed(c, stage_mode ? kProfSweepXStage1D : kProfSweepXRhs,
                 [&] { return launch_sweep_x<T>(c->gi, c->s, x, c->stream); });
  }
  // 2D: the x sweep writes L_x (RHS) or the partial stage (all terms but the y part of L)
  // into R (skipped when dt == 0), then the y sweep adds L_y or its stage multiple.  A
  // stage on a grid with a partial-stage ring runs both sweeps in one banded launch.
  x.out = static_cast<T*>(c->R);
  x.dt = stage_mode ? c->d_dt : nullptr;
  x.un = static_cast<const T*>(un);
  x.a = k.a; x.b = k.b;
  x.stage = stage_mode;
  SweepCall<T> y{};
  y.u = static_cast<const T*>(u);
  y.un = static_cast<const T*>(un);
  y.R = static_cast<const T*>(c->R);
  y.out = static_cast<T*>(out);
  y.dt = stage_mode ? c->d_dt : nullptr;
  y.a = k.a; y.b = k.b;
  y.general = k.general;
  y.e = k.e;
  y.stage = stage_mode;
  y.fallbacks = c->d_fallbacks;
  y.faces = &c->faces;
  y.cstage = k.cstage;
  y.tnow = c->d_t;
  y.status = c->d_err;
  if (stage_mode && k.last && c->fuse_wave) {
    y.wave = c->d_wave;
    y.err = c->d_err;
  }
  if (stage_mode && c->banded)
    return timed(c, kProfStageBand, [&] {
      return launch_stage_band<T>(c->gi, c->s, x, y, static_cast<T*>(c->ring), c->d_band, c->d_err, c->stream);
    });
  cudaError_t e = timed(c, stage_mode ? kProfSweepXLx : kProfSweepXRhs,
                        [&] { return launch_sweep_x<T>(c->gi, c->s, x, c->stream); });
  if (e != cudaSuccess) return e;
  return timed(c, stage_mode ? kProfSweepYStage : kProfSweepYRhs,
               [&] { return launch_sweep_y<T>(c->gi, c->s, y, c->stream); });
}

cudaError_t rhs_into(wcns_ctx* c, const void* u, void* out) {
  StageCoef k{0.0, 1.0, false, 0.0, 0.0, 0.0, nullptr, nullptr, 0.0, false};
  return by_type(c->g.dtype, [&] { return sweeps<double>(c, u, nullptr, out, false, k); },
                 [&] { return sweeps<float>(c, u, nullptr, out, false, k); });
}

cudaError_t stage_coef(wcns_ctx* c, const void* u, const void* un, void* out, const StageCoef& k) {
  return by_type(c->g.dtype, [&] { return sweeps<double>(c, u, un, out, true, k); },
                 [&] { return sweeps<float>(c, u, un, out, true, k); });
}

// TVD-RK3 stage out = a*un + b*(u + dt*L(u)), u at time t0 + cstage * dt.
cudaError_t stage(wcns_ctx* c, const void* u, const void* un, void* out, double a, double b, double cstage,
                  bool last = false) {
  StageCoef k{a, b, false, 0.0, 0.0, 0.0, nullptr, nullptr, cstage, last};
  return stage_coef(c, u, un, out, k);
}

cudaError_t dt_launch(wcns_ctx* c, const void* u, double dt, double t_end, bool maxwave_only,
                      void* copy = nullptr) {
  DtLaunch d{};
  d.u = u;
  d.copy = copy;
  d.cfl = c->p.cfl;
  d.fixed_dt = dt;
  d.t_end = t_end;
  d.use_cfl = dt > 0.0 ? 0 : 1;
  d.gamma = c->p.gamma;
  for (int k = 0; k < 2; ++k) d.adv_wave[k] = fabs(c->p.adv_speed[k]);
  d.partials = c->d_partials;
  d.max_blocks = kMaxRedBlocks;
  d.counter = c->d_counters;
  d.dt_out = c->d_out;
  d.step = c->d_dt;
  d.t = maxwave_only ? nullptr : c->d_t;
  d.steps = c->d_steps;
  d.err = c->d_err;
  d.wave = c->fuse_wave ? c->d_wave : nullptr;
  return timed(c, kProfDt, [&] {
    return by_type(c->g.dtype, [&] { return launch_dt<double>(c->gi, d, c->stream); },
                   [&] { return launch_dt<float>(c->gi, d, c->stream); });
  });
}

// The step record of a step whose CFL maxima the previous step's last stage reduced
// (fused path of 2D Euler grids): the CFL kernel's step computation without reading u.
cudaError_t dt_from_maxima(wcns_ctx* c, double dt, double t_end) {
  DtLaunch d{};
  d.cfl = c->p.cfl;
  d.fixed_dt = dt;
  d.t_end = t_end;
  d.use_cfl = dt > 0.0 ? 0 : 1;
  for (int k = 0; k < 2; ++k) d.adv_wave[k] = fabs(c->p.adv_speed[k]);
  d.step = c->d_dt;
  d.t = c->d_t;
  d.steps = c->d_steps;
  d.err = c->d_err;
  d.wave = c->d_wave;
  return timed(c, kProfDtFused, [&] {
    return by_type(c->g.dtype, [&] { return launch_step_from_maxima<double>(c->gi, d, c->stream); },
                   [&] { return launch_step_from_maxima<float>(c->gi, d, c->stream); });
  });
}

// out = c1 X1 + c2 X2 + b (mu + dt J(u)^T mu), J = dL/du (both sweeps).
template <typename T>
cudaError_t adjoint_stage(wcns_ctx* c, const void* u, const void* mu, const void* X1, double c1, const void* X2,
                          double c2, double b, double dt, void* out) {
  AdjCall<T> a{};
  a.u = static_cast<const T*>(u);
  a.mu = static_cast<const T*>(mu);
  a.X1 = static_cast<const T*>(X1);
  a.X2 = static_cast<const T*>(X2);
  a.c1 = c1; a.c2 = c2; a.b = b; a.dt = dt;
  if (c->g.ndim == 1) {
    a.out = static_cast<T*>(out);
    a.combine = true;
    return timed(c, kProfAdjX, [&] { return launch_adjoint_x<T>(c->gi, c->s, a, c->stream); });
  }
  AdjCall<T> x = a;
  x.out = static_cast<T*>(c->R);
  x.combine = false;
  cudaError_t e = timed(c, kProfAdjX, [&] { return launch_adjoint_x<T>(c->gi, c->s, x, c->stream); });
  if (e != cudaSuccess) return e;
  a.R = static_cast<const T*>(c->R);
  a.out = static_cast<T*>(out);
  a.combine = true;
  return timed(c, kProfAdjY, [&] { return launch_adjoint_y<T>(c->gi, c->s, a, c->stream); });
}

// One TVD-RK3 step on u in place (Shu-Osher form), or one classical RK4 step in the
// form printed as Eq. 16:
//   u1 = u + dt/2 L(u), u2 = u + dt/2 L(u1), u3 = u + dt L(u2),
//   u' = -u/3 + u1/3 + 2 u2/3 + u3/3 + dt/6 L(u3).
//
// src: where the CFL kernel reads u^n; if it is not u, the kernel also copies it into u
// (the host-buffer path reads a mapped host buffer once).  out: where the last stage
// writes u^(n+1) (u itself, or the mapped host buffer).
// from_maxima (2D Euler, a step that follows a step of the same run on the same buffer):
// the step comes from the CFL maxima the previous step's last stage reduced, instead of
// a CFL kernel reading u^n.  On 2D Euler grids every step's last stage reduces them.
cudaError_t rk_step_io(wcns_ctx* c, const void* src, void* u, void* out, double dt, double t_end,
                       bool from_maxima = false, void* s1 = nullptr, void* s2 = nullptr) {
  // s1, s2: where the TVD-RK3 step writes its two inner stage states (default: the
  // context's stage scratch)
  void* u1 = s1 ? s1 : c->u1;
  void* u2 = s2 ? s2 : c->u2;
  cudaError_t e;
  if (from_maxima && c->fuse_wave && src == u) {
    if ((e = dt_from_maxima(c, dt, t_end)) != cudaSuccess) return e;
  } else if ((e = dt_launch(c, src, dt, t_end, false, src != u ? u : nullptr)) != cudaSuccess) {
    return e;
  }
  if (c->p.integrator == WCNS_RK4) {
    StageCoef k1{0.0, 1.0, true, 0.5, 0.0, 0.0, nullptr, nullptr, 0.0, false};
    if ((e = stage_coef(c, u, u, c->u1, k1)) != cudaSuccess) return e;
    StageCoef k2{1.0, 0.0, true, 0.5, 0.0, 0.0, nullptr, nullptr, 0.5, false};
    if ((e = stage_coef(c, c->u1, u, c->u2, k2)) != cudaSuccess) return e;
    StageCoef k3{1.0, 0.0, true, 1.0, 0.0, 0.0, nullptr, nullptr, 0.5, false};
    if ((e = stage_coef(c, c->u2, u, c->u3, k3)) != cudaSuccess) return e;
    StageCoef k4{-1.0 / 3.0, 1.0 / 3.0, true, 1.0 / 6.0, 1.0 / 3.0, 2.0 / 3.0, c->u1, c->u2, 1.0, true};
    return stage_coef(c, c->u3, u, out, k4);
  }
  // stage times t, t + dt, t + dt/2
  if ((e = stage(c, u, nullptr, u1, 0.0, 1.0, 0.0)) != cudaSuccess) return e;
  if ((e = stage(c, u1, u, u2, 0.75, 0.25, 1.0)) != cudaSuccess) return e;
  return stage(c, u2, u, out, 1.0 / 3.0, 2.0 / 3.0, 0.5, true);
}

cudaError_t rk3_step(wcns_ctx* c, void* u, double dt, double t_end, bool from_maxima) {
  return rk_step_io(c, u, u, u, dt, t_end, from_maxima);
}

// Device address of page-locked host memory registered in this context, or nullptr
// (pageable memory, another device's allocation, or a device pointer).
void* mapped_host(const wcns_ctx* c, void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer || a.device != c->device) return nullptr;
  return a.devicePointer;
}

void drop_graph(wcns_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->graph_next) cudaGraphExecDestroy(c->graph_next);
  c->graph = nullptr;
  c->graph_next = nullptr;
  c->graph_u = nullptr;
}

cudaError_t capture_step(wcns_ctx* c, void* u, double dt, double t_end, bool from_maxima, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t body = rk3_step(c, u, dt, t_end, from_maxima);
  e = cudaStreamEndCapture(c->stream, &g);
  if (body != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return body;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) *out = nullptr;
  return e;
}

// Graphs of one step on u: the first step of a call (CFL kernel) and, on 2D Euler grids,
// the following ones (step from the maxima the previous step's last stage reduced).
cudaError_t build_graph(wcns_ctx* c, void* u, double dt, double t_end) {
  drop_graph(c);
  cudaError_t e = capture_step(c, u, dt, t_end, false, &c->graph);
  if (e == cudaSuccess && c->fuse_wave) e = capture_step(c, u, dt, t_end, true, &c->graph_next);
  if (e != cudaSuccess) {
    drop_graph(c);
    return e;
  }
  c->graph_u = u;
  c->graph_dt = dt;
  c->graph_tend = t_end;
  return cudaSuccess;
}

// nsteps steps of u.  continuing: the previous step of this run on u was the last one
// enqueued (its last stage reduced the CFL maxima of u), so on 2D Euler grids the first
// step also takes its step from them.
cudaError_t step_run(wcns_ctx* c, void* u, double dt, int32_t nsteps, double t_end, bool continuing) {
  // Replaying a captured step graph needs a capturable stream (not the legacy default);
  // per-kernel timing launches directly.
  if (c->stream != nullptr && nsteps >= 2 && !c->prof_on) {
    if (!c->graph || c->graph_u != u || c->graph_dt != dt || c->graph_tend != t_end) {
      cudaError_t e = build_graph(c, u, dt, t_end);
      if (e != cudaSuccess) return e;
    }
    for (int32_t k = 0; k < nsteps; ++k) {
      cudaGraphExec_t g = (c->fuse_wave && (k > 0 || continuing)) ? c->graph_next : c->graph;
      cudaError_t e = cudaGraphLaunch(g, c->stream);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  for (int32_t k = 0; k < nsteps; ++k) {
    cudaError_t e = rk3_step(c, u, dt, t_end, k > 0 || continuing);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

namespace {
__global__ void reciprocal_f64_kernel(const double* x, double* out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = Num<double>::rcp_(x[i]);
}
}  // namespace

namespace {
// Options the hand-written adjoint covers.
bool adjoint_supported(const wcns_ctx* c) {
  const wcns_params& p = c->p;
  return p.system == WCNS_EULER && p.flux == WCNS_FLUX_LLF_FROZEN && p.weights != WCNS_W_M &&
         p.integrator == WCNS_RK3 && p.family == WCNS_FAMILY_WCNS && !c->faces.active;
}

// The three reverse RK stages of one TVD-RK3 step, at the step's stage states u_n, u1, u2.
wcns_status adjoint_from_stages(wcns_ctx* c, const void* u_n, const void* u1, const void* u2, double dt,
                                     const void* lam_np1, void* lam_n) {
  const size_t bytes = c->nelem * c->elem;
  if (!c->adj1) WCNS_TRY(cudaMalloc(&c->adj1, bytes));
  if (!c->adj2) WCNS_TRY(cudaMalloc(&c->adj2, bytes));
  // reverse of u' = 1/3 u + 2/3 (u2 + dt L(u2)), u2 = 3/4 u + 1/4 (u1 + dt L(u1)), u1 = u + dt L(u):
  //   a2 = 2/3 (lam + dt J(u2)^T lam)
  //   a1 = 1/4 (a2 + dt J(u1)^T a2)
  //   lam_n = 1/3 lam + 3/4 a2 + (a1 + dt J(u)^T a1)
  auto reverse_stage = [&](const void* u, const void* mu, const void* X1, double c1, const void* X2, double c2,
                           double b, void* out) -> cudaError_t {
    return by_type(
        c->g.dtype,
        [&] { return adjoint_stage<double>(c, u, mu, X1, c1, X2, c2, b, dt, out); },
        [&] { return adjoint_stage<float>(c, u, mu, X1, c1, X2, c2, b, dt, out); });
  };
  WCNS_TRY(reverse_stage(u2, lam_np1, nullptr, 0.0, nullptr, 0.0, 2.0 / 3.0, c->adj1));
  WCNS_TRY(reverse_stage(u1, c->adj1, nullptr, 0.0, nullptr, 0.0, 0.25, c->adj2));
  WCNS_TRY(reverse_stage(u_n, c->adj2, lam_np1, 1.0 / 3.0, c->adj1, 0.75, 1.0, lam_n));
  return WCNS_OK;
}

}  // namespace

extern "C" {

const char* wcns_status_string(wcns_status s) {
  switch (s) {
    case WCNS_OK: return "ok";
    case WCNS_ERR_ARG: return "invalid argument";
    case WCNS_ERR_CUDA: return "CUDA runtime error";
    case WCNS_ERR_NONPHYSICAL: return "non-physical state (rho <= 0, p <= 0 or NaN)";
    case WCNS_ERR_TIMEOUT: return "bounded device wait expired";
    case WCNS_ERR_UNSUPPORTED: return "unsupported option combination";
    case WCNS_ERR_NOMEM: return "device allocation failed";
  }
  return "unknown status";
}

wcns_status wcns_default_params(int32_t system, int32_t dtype, wcns_params* p) {
  if (!p || (system != WCNS_ADVECTION && system != WCNS_EULER) || (dtype != WCNS_F64 && dtype != WCNS_F32))
    return WCNS_ERR_ARG;
  std::memset(p, 0, sizeof(*p));
  p->system = system;
  p->weights = WCNS_W_FE;
  p->flux = WCNS_FLUX_HLLC;
  p->characteristic = 1;
  p->z_p = 1;
  p->renorm = 1;
  p->adv_speed[0] = 1.0;
  p->gamma = 1.4;
  p->eps = dtype == WCNS_F64 ? 1e-40 : 1e-30;
  p->xi = 1e6;
  p->kappa = 0.5;
  p->cv = 1e-3;
  p->cfl = 0.5;
  p->harten = 0.1;
  return WCNS_OK;
}

wcns_status wcns_init(const wcns_grid* grid, const wcns_params* params, void* stream, wcns_ctx** out) {
  if (!out) return WCNS_ERR_ARG;
  *out = nullptr;
  if (!grid || !params) return WCNS_ERR_ARG;
  const wcns_grid& g = *grid;
  if (g.nvar != 1 && g.nvar != 3 && g.nvar != 4) return WCNS_ERR_ARG;
  if (check_grid_layout(g) != WCNS_OK) return WCNS_ERR_ARG;
  for (int d = 0; d < g.ndim; ++d) {
    if (!(g.hi[d] > g.lo[d])) return WCNS_ERR_ARG;
    if (g.bc[d] != WCNS_BC_PERIODIC && g.bc[d] != WCNS_BC_TRANSMISSIVE) return WCNS_ERR_ARG;
  }
  wcns_status st = check_params(params, g.dtype, g.nvar, g.ndim);
  if (st != WCNS_OK) return st;

  wcns_ctx* c = new (std::nothrow) wcns_ctx();
  if (!c) return WCNS_ERR_NOMEM;
  c->g = g;
  c->p = *params;
  c->s = make_scheme(params);
  c->gi.ndim = g.ndim;
  c->gi.nvar = g.nvar;
  c->gi.nx = g.nx;
  c->gi.ny = g.ny;
  c->gi.pitch = g.pitch;
  c->gi.bc[0] = g.bc[0];
  c->gi.bc[1] = g.ndim == 2 ? g.bc[1] : WCNS_BC_PERIODIC;
  c->gi.h[0] = (g.hi[0] - g.lo[0]) / (double)g.nx;
  c->gi.h[1] = g.ndim == 2 ? (g.hi[1] - g.lo[1]) / (double)g.ny : 1.0;
  c->stream = static_cast<cudaStream_t>(stream);
  c->elem = g.dtype == WCNS_F64 ? 8 : 4;
  c->fuse_wave = g.ndim == 2 && g.nvar == 4;
  c->nelem = (size_t)g.nvar * (size_t)g.ny * (size_t)g.pitch;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess)
    e = by_type(g.dtype, [&] { return configure_kernels<double>(g.nvar); },
                [&] { return configure_kernels<float>(g.nvar); });
  const size_t bytes = c->nelem * c->elem;
  if (e == cudaSuccess) e = cudaMalloc(&c->u1, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->u2, bytes);
  if (e == cudaSuccess && g.ndim == 2) e = cudaMalloc(&c->R, bytes);
  if (e == cudaSuccess && params->integrator == WCNS_RK4) e = cudaMalloc(&c->u3, bytes);
  if (e == cudaSuccess && c->fuse_wave)
    e = cudaMalloc(reinterpret_cast<void**>(&c->d_wave), sizeof(unsigned long long) * 2 * kWaveSlots);
  const size_t scal_bytes = 4096 + sizeof(double) * 2 * kMaxRedBlocks;
  if (e == cudaSuccess) e = cudaMalloc(&c->scal, scal_bytes);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->scal, 0, scal_bytes, c->stream);
  if (e == cudaSuccess && c->fuse_wave)
    e = cudaMemsetAsync(c->d_wave, 0, sizeof(unsigned long long) * 2 * kWaveSlots, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    wcns_destroy(c);
    return from_cuda(e);
  }
  char* b = static_cast<char*>(c->scal);
  c->d_dt = reinterpret_cast<StepDt*>(b + 256);
  c->d_t = reinterpret_cast<double*>(b + 8);
  c->d_steps = reinterpret_cast<long long*>(b + 16);
  c->d_err = reinterpret_cast<int*>(b + 24);
  c->d_fallbacks = reinterpret_cast<unsigned long long*>(b + 32);
  c->d_counters = reinterpret_cast<unsigned int*>(b + 64);
  c->d_out = reinterpret_cast<double*>(b + 128);
  c->d_partials = reinterpret_cast<double*>(b + 4096);
  c->d_band = reinterpret_cast<unsigned*>(b + 1024);  // kBandCounterWords (zeroed above)
  c->banded = false;
  *out = c;
  return WCNS_OK;
}

wcns_status wcns_rhs(wcns_ctx* c, const void* u, void* dudt) {
  if (!c || !u || !dudt || !aligned16(u) || !aligned16(dudt)) return WCNS_ERR_ARG;
  const char* a = static_cast<const char*>(u);
  const char* d = static_cast<const char*>(dudt);
  const size_t bytes = c->nelem * c->elem;
  if (a < d + bytes && d < a + bytes) return WCNS_ERR_ARG;  // must not overlap
  return from_cuda(rhs_into(c, u, dudt));
}

wcns_status wcns_step(wcns_ctx* c, void* u, double dt, int32_t nsteps, double t_end) {
  if (!c || !u || !aligned16(u) || nsteps < 0) return WCNS_ERR_ARG;
  if (dt != dt || t_end != t_end) return WCNS_ERR_ARG;
  if (nsteps == 0) return WCNS_OK;
  return from_cuda(step_run(c, u, dt, nsteps, t_end, false));
}

wcns_status wcns_step_host(wcns_ctx* c, void* u_host, double dt, int32_t nsteps, double t_end) {
  if (!c || !u_host || nsteps < 0) return WCNS_ERR_ARG;
  if (dt != dt || t_end != t_end) return WCNS_ERR_ARG;
  const size_t bytes = c->nelem * c->elem;
  if (!c->host_state) WCNS_TRY(cudaMalloc(&c->host_state, bytes));
  if (nsteps == 0) return WCNS_OK;
  void* hd = mapped_host(c, u_host);
  if (!hd || !aligned16(hd) || c->g.nvar == 1) {
    WCNS_TRY(cudaMemcpyAsync(c->host_state, u_host, bytes, cudaMemcpyHostToDevice, c->stream));
    wcns_status s = wcns_step(c, c->host_state, dt, nsteps, t_end);
    if (s != WCNS_OK) return s;
    WCNS_TRY(cudaMemcpyAsync(u_host, c->host_state, bytes, cudaMemcpyDeviceToHost, c->stream));
    WCNS_TRY(cudaStreamSynchronize(c->stream));
    return WCNS_OK;
  }
  // Page-locked host buffer: the first step's CFL kernel reads it through its device
  // address and writes the device working copy as it goes (no separate copy in).  With
  // one step the last stage writes u^(n+1) straight into the host buffer; with more, the
  // remaining steps run on the working copy and one copy brings it back (a step frozen
  // at t_end writes nothing, so the last stage cannot stand in for that copy).
  if (nsteps == 1) {
    WCNS_TRY(rk_step_io(c, hd, c->host_state, hd, dt, t_end));
  } else {
    WCNS_TRY(rk_step_io(c, hd, c->host_state, c->host_state, dt, t_end));
    WCNS_TRY(step_run(c, c->host_state, dt, nsteps - 1, t_end, true));
    WCNS_TRY(cudaMemcpyAsync(u_host, c->host_state, bytes, cudaMemcpyDeviceToHost, c->stream));
  }
  WCNS_TRY(cudaStreamSynchronize(c->stream));
  return WCNS_OK;
}

wcns_status wcns_set_time(wcns_ctx* c, double t) {
  if (!c || t != t) return WCNS_ERR_ARG;
  WCNS_TRY(cudaMemcpyAsync(c->d_t, &t, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  WCNS_TRY(cudaMemsetAsync(c->d_steps, 0, sizeof(long long), c->stream));
  WCNS_TRY(cudaStreamSynchronize(c->stream));
  return WCNS_OK;
}

wcns_status wcns_get_time(wcns_ctx* c, double* t, int64_t* steps) {
  if (!c) return WCNS_ERR_ARG;
  double tt = 0.0;
  long long ss = 0;
  WCNS_TRY(cudaMemcpyAsync(&tt, c->d_t, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  WCNS_TRY(cudaMemcpyAsync(&ss, c->d_steps, sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
  WCNS_TRY(cudaStreamSynchronize(c->stream));
  if (t) *t = tt;
  if (steps) *steps = (int64_t)ss;
  return WCNS_OK;
}

wcns_status wcns_reduce(wcns_ctx* c, const void* a, const void* b, int32_t what, double* out) {
  if (!c || !a || !out || !aligned16(a) || (b && !aligned16(b))) return WCNS_ERR_ARG;
  if (what < WCNS_REDUCE_SUM || what > WCNS_REDUCE_MAXWAVE) return WCNS_ERR_ARG;
  int nout;
  if (what == WCNS_REDUCE_MAXWAVE) {
    WCNS_TRY(dt_launch(c, a, 0.0, 0.0, true));
    nout = c->g.ndim;
  } else {
    WCNS_TRY(timed(c, kProfReduce, [&] {
      return by_type(
          c->g.dtype,
          [&] { return launch_reduce<double>(c->gi, a, b, what, c->d_partials, 2 * kMaxRedBlocks, c->d_counters, c->d_out, c->stream); },
          [&] { return launch_reduce<float>(c->gi, a, b, what, c->d_partials, 2 * kMaxRedBlocks, c->d_counters, c->d_out, c->stream); });
    }));
    nout = c->g.nvar;
  }
  WCNS_TRY(cudaMemcpyAsync(out, c->d_out, sizeof(double) * nout, cudaMemcpyDeviceToHost, c->stream));
  WCNS_TRY(cudaStreamSynchronize(c->stream));
  if (what == WCNS_REDUCE_MAXWAVE && c->p.system == WCNS_ADVECTION)
    for (int d = 0; d < nout; ++d) out[d] = fabs(c->p.adv_speed[d]);
  return WCNS_OK;
}

wcns_status wcns_weight_hist(wcns_ctx* c, const void* u, int32_t nbins, uint64_t* hist) {
  if (!c || !u || !hist || !aligned16(u) || (reinterpret_cast<uintptr_t>(hist) & 7u)) return WCNS_ERR_ARG;
  if (nbins < 1 || nbins > (1 << 20)) return WCNS_ERR_ARG;
  unsigned long long* h = reinterpret_cast<unsigned long long*>(hist);
  WCNS_TRY(by_type(
      c->g.dtype, [&] { return launch_weight_hist<double>(c->gi, c->s, c->faces, c->d_t, u, nbins, h, c->stream); },
      [&] { return launch_weight_hist<float>(c->gi, c->s, c->faces, c->d_t, u, nbins, h, c->stream); }));
  return WCNS_OK;
}

wcns_status wcns_set_faces(wcns_ctx* c, const wcns_faces* f) {
  if (!c) return WCNS_ERR_ARG;
  Faces<double> r{};
  if (f) {
    for (int k = 0; k < 4; ++k)
      if (f->reserved[k] != 0) return WCNS_ERR_ARG;
    for (int k = 0; k < 4; ++k) {
      const int t = f->type[k];
      if (t < WCNS_FACE_GRID || t > WCNS_FACE_SHOCK) return WCNS_ERR_ARG;
      if (t == WCNS_FACE_GRID) continue;
      const int dir = k / 2;
      if (dir >= c->g.ndim) return WCNS_ERR_ARG;              // no y faces on 1D grids
      if (c->g.bc[dir] == WCNS_BC_PERIODIC) return WCNS_ERR_ARG;  // periodic lines have no faces
      if (t >= WCNS_FACE_WALL && c->p.system != WCNS_EULER) return WCNS_ERR_UNSUPPORTED;
      r.type[k] = t;
      r.active = 1;
    }
    const double* st[2] = {f->state_a, f->state_b};
    for (int q = 0; q < 2; ++q) {
      const double rho = st[q][0], u = st[q][1], v = st[q][2], p = st[q][3];
      double* U = q == 0 ? r.ua : r.ub;
      if (r.active && c->p.system == WCNS_EULER && !(rho > 0.0 && p > 0.0)) {
        bool used = false;
        for (int k = 0; k < 4; ++k)
          used = used || (q == 0 ? r.type[k] >= WCNS_FACE_FIXED : r.type[k] == WCNS_FACE_SHOCK);
        if (used) return WCNS_ERR_ARG;
      }
      const double E = p / (c->p.gamma - 1.0) + 0.5 * rho * (u * u + (c->g.nvar == 4 ? v * v : 0.0));
      U[0] = rho;
      U[1] = rho * u;
      if (c->g.nvar == 4) { U[2] = rho * v; U[3] = E; } else { U[2] = E; U[3] = 0.0; }
    }
    r.wall_x = f->wall_x;
    r.x0 = f->shock_x0;
    r.dxdy = f->shock_dxdy;
    r.speed = f->shock_speed;
    r.lo_x = c->g.lo[0];
    r.lo_y = c->g.lo[1];
    r.hx = c->gi.h[0];
    r.hy = c->gi.h[1];
  }
  c->faces = r;
  drop_graph(c);  // captured steps hold the old face arguments
  return WCNS_OK;
}

wcns_status wcns_selftest_waits(wcns_ctx* c, int32_t* gave_up) {
  if (!c || !gave_up) return WCNS_ERR_ARG;
  // word 0 of the banded-stage counters is zeroed at init and never written: a counter
  // that nothing increments; the results go to the context's scalar outputs
  int* d_res = reinterpret_cast<int*>(c->d_out);
  WCNS_TRY(launch_wait_selftest(c->d_band, c->d_err, d_res, c->stream));
  int h[2] = {0, 0};
  WCNS_TRY(cudaMemcpyAsync(h, d_res, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  WCNS_TRY(cudaStreamSynchronize(c->stream));
  gave_up[0] = h[0];
  gave_up[1] = h[1];
  return WCNS_OK;
}

wcns_status wcns_set_stage_form(wcns_ctx* c, int32_t banded) {
  if (!c) return WCNS_ERR_ARG;
  if (banded) {
    if (!by_type_bool(c->g.dtype, band_applies<double>(c->gi, c->s), band_applies<float>(c->gi, c->s)))
      return WCNS_ERR_UNSUPPORTED;
    if (!c->ring) WCNS_TRY(cudaMalloc(&c->ring, band_ring_bytes_of(c->gi, c->elem)));
  }
  if (c->banded != (banded != 0)) drop_graph(c);  // captured steps hold the other form
  c->banded = banded != 0;
  return WCNS_OK;
}

wcns_status wcns_adjoint_step(wcns_ctx* c, const void* u_n, double dt, const void* lam_np1, void* lam_n) {
  if (!c || !u_n || !lam_np1 || !lam_n || !aligned16(u_n) || !aligned16(lam_np1) || !aligned16(lam_n))
    return WCNS_ERR_ARG;
  if (u_n == lam_np1 || u_n == lam_n) return WCNS_ERR_ARG;  // the checkpoint is read after lam_n is written
  if (!(dt > 0.0)) return WCNS_ERR_ARG;
  if (!adjoint_supported(c)) return WCNS_ERR_UNSUPPORTED;
  // stage states of the forward step, recomputed from the checkpoint u_n
  const StepDt step{dt, 0.0, (float)dt, 0};
  WCNS_TRY(cudaMemcpyAsync(c->d_dt, &step, sizeof(step), cudaMemcpyHostToDevice, c->stream));
  WCNS_TRY(stage(c, u_n, nullptr, c->u1, 0.0, 1.0, 0.0));
  WCNS_TRY(stage(c, c->u1, u_n, c->u2, 0.75, 0.25, 1.0));
  return adjoint_from_stages(c, u_n, c->u1, c->u2, dt, lam_np1, lam_n);
}

wcns_status wcns_adjoint_step_stages(wcns_ctx* c, const void* u_n, const void* u1, const void* u2, double dt,
                                     const void* lam_np1, void* lam_n) {
  if (!c || !u_n || !u1 || !u2 || !lam_np1 || !lam_n || !aligned16(u_n) || !aligned16(u1) || !aligned16(u2) ||
      !aligned16(lam_np1) || !aligned16(lam_n))
    return WCNS_ERR_ARG;
  for (const void* q : {u_n, u1, u2})
    if (q == lam_np1 || q == lam_n) return WCNS_ERR_ARG;  // the stage states are read after lam_n is written
  if (!(dt > 0.0)) return WCNS_ERR_ARG;
  if (!adjoint_supported(c)) return WCNS_ERR_UNSUPPORTED;
  return adjoint_from_stages(c, u_n, u1, u2, dt, lam_np1, lam_n);
}

wcns_status wcns_step_stages(wcns_ctx* c, void* u, double dt, void* u1_out, void* u2_out) {
  if (!c || !u || !u1_out || !u2_out || !aligned16(u) || !aligned16(u1_out) || !aligned16(u2_out)) return WCNS_ERR_ARG;
  if (u1_out == u || u2_out == u || u1_out == u2_out) return WCNS_ERR_ARG;
  if (!(dt > 0.0)) return WCNS_ERR_ARG;
  if (c->p.integrator != WCNS_RK3) return WCNS_ERR_UNSUPPORTED;
  // the first step of a call: the CFL kernel writes the step record (fixed dt) and
  // advances the device time, as wcns_step(ctx, u, dt, 1, 0) does
  return from_cuda(rk_step_io(c, u, u, u, dt, 0.0, false, u1_out, u2_out));
}

wcns_status wcns_reciprocal_f64(const double* x, double* out, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !out))) return WCNS_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(x) & 7u) || (reinterpret_cast<uintptr_t>(out) & 7u)) return WCNS_ERR_ARG;
  if (n == 0) return WCNS_OK;
  const int64_t blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
  reciprocal_f64_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(x, out, n);
  return from_cuda(cudaGetLastError());
}

wcns_status wcns_sync_status(wcns_ctx* c, int64_t* nonphysical) {
  if (!c) return WCNS_ERR_ARG;
  int err = 0;
  unsigned long long fb = 0;
  WCNS_TRY(cudaMemcpyAsync(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  WCNS_TRY(cudaMemcpyAsync(&fb, c->d_fallbacks, sizeof(fb), cudaMemcpyDeviceToHost, c->stream));
  WCNS_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
  WCNS_TRY(cudaMemsetAsync(c->d_fallbacks, 0, sizeof(fb), c->stream));
  WCNS_TRY(cudaStreamSynchronize(c->stream));
  if (nonphysical) *nonphysical = (int64_t)fb;
  if (err & 2) return WCNS_ERR_TIMEOUT;
  if (err & 1) return WCNS_ERR_NONPHYSICAL;
  return WCNS_OK;
}

wcns_status wcns_profile_enable(wcns_ctx* c, int32_t on) {
  if (!c) return WCNS_ERR_ARG;
  c->prof_on = on != 0;
  c->prof_used = 0;
  return WCNS_OK;
}

wcns_status wcns_profile_read(wcns_ctx* c, int32_t max_entries, char* names, int64_t* launches, double* ms,
                              int32_t* n_entries) {
  if (!c || max_entries < kProfCount || !names || !launches || !ms || !n_entries) return WCNS_ERR_ARG;
  WCNS_TRY(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < kProfCount; ++k) {
    std::snprintf(names + 48 * k, 48, "%s", kProfNames[k]);
    launches[k] = 0;
    ms[k] = 0.0;
  }
  for (size_t i = 0; i < c->prof_used; ++i) {
    float t = 0.f;
    WCNS_TRY(cudaEventElapsedTime(&t, c->prof[i].a, c->prof[i].b));
    launches[c->prof[i].kind] += 1;
    ms[c->prof[i].kind] += t;
  }
  c->prof_used = 0;
  *n_entries = kProfCount;
  return WCNS_OK;
}

void wcns_destroy(wcns_ctx* c) {
  if (!c) return;
  if (c->stream || c->u1) cudaStreamSynchronize(c->stream);
  for (auto& ev : c->prof) {
    cudaEventDestroy(ev.a);
    cudaEventDestroy(ev.b);
  }
  drop_graph(c);
  if (c->u1) cudaFree(c->u1);
  if (c->u2) cudaFree(c->u2);
  if (c->u3) cudaFree(c->u3);
  if (c->R) cudaFree(c->R);
  if (c->ring) cudaFree(c->ring);
  if (c->host_state) cudaFree(c->host_state);
  if (c->adj1) cudaFree(c->adj1);
  if (c->adj2) cudaFree(c->adj2);
  if (c->scal) cudaFree(c->scal);
  if (c->d_wave) cudaFree(c->d_wave);
  delete c;
}

// Batched problems: implemented in wcns_batch.cu.

}  // extern "C"
