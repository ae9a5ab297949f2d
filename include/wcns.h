/*
 * wcns.h -- C ABI of the WCNS-FE solver library (libwcns.so) for one GB300 GPU.
 *
 * The library evaluates the right-hand side of the semi-discrete conservation law
 * du_i/dt = -df/dx|_i (Sec. 2, Eq. 1-2) with the filtered embedded weighted compact
 * nonlinear scheme of Liu, Min, Cai, Ma and Yan (arXiv 2306.09760) and advances it
 * with third-order TVD Runge-Kutta.  Per sweep direction and interface i+1/2:
 *   (a) project the six stencil states U_{i-2..i+3} onto characteristic fields with
 *       Roe-averaged eigenvectors (Euler), or use them as they are (advection);
 *   (b) interpolate each field to the midpoint from the sub-stencils S0, S1, S2
 *       (Eq. 5), with smoothness indicators (Eq. 9-10), JS / Z / M weights
 *       (Eq. 11-15) and the FE mapping function (Eq. 20-21, Table 2) or its PFE
 *       switch (App. A), for the left state and the mirrored right state;
 *   (c) form the midpoint flux with an approximate Riemann solver (Eq. 6);
 *   (d) take the sixth-order midpoint flux difference (Eq. 3);
 *   (e) apply a TVD-RK3 stage.
 *
 * Conventions shared by every entry point
 *   - Arrays ("state buffers") live in device memory unless a function says "host".
 *     The caller owns them; the library never frees or retains them past the call's
 *     stream work.  Layout: element (v, j, i) of a grid buffer is at offset
 *     (v * ny + j) * pitch + i elements -- structure of arrays, one plane per
 *     conserved variable v, rows j of `pitch` elements, cells i contiguous.
 *     Element type: double (WCNS_F64) or float (WCNS_F32), fixed per context.
 *     Device pointers must be 16-byte aligned.
 *   - Conserved variables: advection (u); Euler 1D (rho, rho u, E); Euler 2D
 *     (rho, rho u, rho v, E), ideal gas p = (gamma - 1)(E - rho |v|^2 / 2).
 *   - Ghost cells are not stored: boundary conditions are applied by index
 *     arithmetic (periodic: modulo; transmissive: the nearest interior cell).
 *   - All work is enqueued asynchronously on the context's CUDA stream (the stream
 *     handle passed at creation; NULL = the legacy default stream).  Functions that
 *     return results to the host synchronise that stream and say so.
 *   - Errors: argument errors are returned at once and nothing is enqueued.  Errors
 *     the device detects (non-physical state, an expired bounded wait) are sticky:
 *     they are recorded in device memory and returned by wcns_sync_status().  No
 *     C++ exception crosses this interface and no kernel traps.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef WCNS_H_
#define WCNS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  WCNS_OK = 0,
  WCNS_ERR_ARG = 1,          /* invalid argument (null, size, alignment, enum value) */
  WCNS_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  WCNS_ERR_NONPHYSICAL = 3,  /* a cell state had rho <= 0, p <= 0 or NaN (sticky) */
  WCNS_ERR_TIMEOUT = 4,      /* a bounded device-side wait expired (sticky) */
  WCNS_ERR_UNSUPPORTED = 5,  /* option combination not implemented */
  WCNS_ERR_NOMEM = 6         /* device allocation failed */
} wcns_status;

enum { WCNS_F64 = 0, WCNS_F32 = 1 };                            /* element type */
enum { WCNS_BC_PERIODIC = 0, WCNS_BC_TRANSMISSIVE = 1 };        /* boundary per direction */
enum { WCNS_ADVECTION = 0, WCNS_EULER = 1 };                    /* equation system */
/* Weights: JS (Eq. 11), Z (Eq. 14-15), FE = Z weights mapped by Eq. 20 and
 * renormalised, PFE = FE with the App. A switch, M = Henrick mapping (Eq. 12-13). */
enum { WCNS_W_JS = 0, WCNS_W_Z = 1, WCNS_W_FE = 2, WCNS_W_PFE = 3, WCNS_W_M = 4 };
/* Midpoint flux (Eq. 6; the paper names no solver): local Lax-Friedrichs, Roe with
 * Harten's entropy fix on the acoustic fields, HLLC with Einfeldt speeds, and
 * Lax-Friedrichs with a frozen dissipation speed alpha[d] (smooth; for adjoints). */
enum { WCNS_FLUX_LLF = 0, WCNS_FLUX_ROE = 1, WCNS_FLUX_HLLC = 2, WCNS_FLUX_LLF_FROZEN = 3 };
enum { WCNS_REDUCE_SUM = 0, WCNS_REDUCE_L1 = 1, WCNS_REDUCE_LINF = 2, WCNS_REDUCE_MAXWAVE = 3 };
/* Time integrator: third-order TVD Runge-Kutta (Shu-Osher form; default) or the
 * classical fourth-order Runge-Kutta the paper uses, in the form printed as Eq. 16. */
enum { WCNS_RK3 = 0, WCNS_RK4 = 1 };
/* Scheme family: the WCNS of Sec. 2-3 (midpoint interpolation of the state, a Riemann
 * solver, the sixth-order difference of Eq. 3), or the fifth-order finite-difference
 * WENO of App. B (Lax-Friedrichs split fluxes reconstructed with the same Z/FE weights,
 * the FE map taking the control rows of Table B.2, and the difference
 * -(F_{i+1/2} - F_{i-1/2}) / h).  `flux` is ignored by the WENO family. */
enum { WCNS_FAMILY_WCNS = 0, WCNS_FAMILY_WENO = 1 };

/* Grid descriptor (Sec. 2: uniform cells, h = (hi - lo) / n per direction). */
typedef struct {
  int32_t ndim;      /* 1 or 2 */
  int32_t nvar;      /* 1 (advection), 3 (Euler, ndim 1), 4 (Euler, ndim 2) */
  int32_t dtype;     /* WCNS_F64 or WCNS_F32 */
  int32_t reserved;  /* must be 0 */
  int64_t nx, ny;    /* cells; 1 <= nx, ny <= 2^26.  ndim = 1 with ny > 1 holds ny
                        independent lines of nx cells (no coupling between rows). */
  int64_t pitch;     /* elements per row; pitch >= nx and pitch % 32 == 0 */
  double lo[2], hi[2];
  int32_t bc[2];     /* WCNS_BC_* for x and y */
} wcns_grid;

/* Scheme parameters.  wcns_default_params() fills the defaults named below. */
typedef struct {
  int32_t system;          /* WCNS_ADVECTION or WCNS_EULER */
  int32_t weights;         /* WCNS_W_*; default FE */
  int32_t flux;            /* WCNS_FLUX_*; default HLLC */
  int32_t characteristic;  /* 1: interpolate characteristic variables (default); 0: conserved */
  int32_t z_p;             /* Z-weight exponent p of Eq. 14, 1 or 2; default 1 */
  int32_t renorm;          /* 1: renormalise the mapped weights (default) */
  int32_t integrator;      /* WCNS_RK3 (default) or WCNS_RK4 (wcns_step only) */
  int32_t family;          /* WCNS_FAMILY_WCNS (default) or WCNS_FAMILY_WENO */
  double adv_speed[2];     /* advection speed per direction (advection only) */
  double gamma;            /* ratio of specific heats; default 1.4 */
  double eps;              /* epsilon of Eq. 11 / Eq. 14; default 1e-40 (F64), 1e-30 (F32) */
  double xi, kappa;        /* steepness and null-point parameters of Eq. 20; default 1e6, 0.5 */
  double cv;               /* PFE switch width (App. A); default 1e-3 */
  double cfl;              /* CFL number for automatic steps; default 0.5 */
  double alpha[2];         /* frozen Lax-Friedrichs speeds (WCNS_FLUX_LLF_FROZEN) */
  double harten;           /* Roe entropy-fix width delta = harten * (|u| + c); default 0.1 */
} wcns_params;

/* Boundary faces (Sec. 4.3) beyond the grid's periodic / transmissive lines, for the
 * faces x-lo, x-hi, y-lo, y-hi.  Ghost values are taken at the ghost cell's centre
 * (lo + (i + 1/2) h) and, for the moving shock, at the time of the state the RK stage
 * reads (t, t + dt, t + dt/2 for TVD-RK3; t, t + dt/2, t + dt/2, t + dt for RK4):
 *   WCNS_FACE_GRID            the direction's bc (default)
 *   WCNS_FACE_TRANSMISSIVE    zero-gradient copy of the edge cell (outflow)
 *   WCNS_FACE_WALL            inviscid wall: mirror cell with the normal momentum reversed
 *   WCNS_FACE_FIXED           state_a (inflow)
 *   WCNS_FACE_FIXED_THEN_WALL state_a where x < wall_x, a wall beyond (y faces)
 *   WCNS_FACE_SHOCK           state_a where x < shock_x0 + (y + shock_speed t) shock_dxdy,
 *                             state_b beyond (the exact motion of an oblique shock)
 * States are primitive (rho, u, v, p); v is ignored on 1D grids. */
enum { WCNS_FACE_GRID = 0, WCNS_FACE_TRANSMISSIVE = 1, WCNS_FACE_WALL = 2, WCNS_FACE_FIXED = 3,
       WCNS_FACE_FIXED_THEN_WALL = 4, WCNS_FACE_SHOCK = 5 };
typedef struct {
  int32_t type[4];
  int32_t reserved[4];     /* must be 0 */
  double state_a[4], state_b[4];
  double wall_x;
  double shock_x0, shock_dxdy, shock_speed;
} wcns_faces;

typedef struct wcns_ctx wcns_ctx;
typedef struct wcns_batch wcns_batch;

/* Fills *p with the defaults for `system` and element type `dtype`.  Returns
 * WCNS_ERR_ARG on a null pointer or unknown enum. */
wcns_status wcns_default_params(int32_t system, int32_t dtype, wcns_params* p);

/* Creates a context for one grid.  Validates *grid and *params, copies them, and
 * allocates the context's own device scratch: two stage states (2 x nvar*ny*pitch
 * elements), one x-sweep RHS plane set (2D), the device time and step size, and
 * reduction partials.  `stream` is a cudaStream_t (NULL: default stream).
 * Errors: WCNS_ERR_ARG (invalid descriptor), WCNS_ERR_UNSUPPORTED (nvar does not
 * match system/ndim), WCNS_ERR_NOMEM, WCNS_ERR_CUDA.  On error *out is NULL. */
wcns_status wcns_init(const wcns_grid* grid, const wcns_params* params, void* stream,
                      wcns_ctx** out);

/* dudt = L(u) = -(dF/dx + dG/dy), Eq. 2-3, steps (a)-(d) of the header comment.
 * u and dudt: device grid buffers; they must not overlap. */
wcns_status wcns_rhs(wcns_ctx* ctx, const void* u, void* dudt);

/* Advances u in place by nsteps TVD-RK3 steps (Shu-Osher form):
 *   u1 = u + dt L(u),  u2 = 3/4 u + 1/4 (u1 + dt L(u1)),  u <- 1/3 u + 2/3 (u2 + dt L(u2)),
 * or, with integrator WCNS_RK4, classical RK4 steps written as in Eq. 16 (one more
 * stage state of scratch, allocated by wcns_init).
 * dt > 0: fixed step.  dt <= 0: each step takes dt = cfl / sum_d(max(|u_d| + c) / h_d)
 * (advection: |a_d| for max(|u_d| + c)), reduced on the device, never read back.  On
 * 2D Euler grids the first step of a call reduces the maxima from u, and each step's
 * last RK stage reduces them from the state it writes for the step after it (the same
 * values, without a separate read of u).
 * t_end > 0: each step is clipped so the device time t never passes t_end; once t
 * reaches t_end further steps do nothing.  The device time starts at 0 (see
 * wcns_set_time) and is read with wcns_get_time.  Asynchronous. */
wcns_status wcns_step(wcns_ctx* ctx, void* u, double dt, int32_t nsteps, double t_end);

/* wcns_step on a HOST buffer u_host (same layout), all on the context stream; returns
 * once u_host holds the result.  Page-locked memory of the context's device (e.g.
 * cudaHostAlloc) with a 16-byte aligned device address and nvar > 1: the first step's
 * CFL kernel reads u_host through that address and fills the context's device working
 * copy as it goes; with nsteps == 1 the last RK stage writes u^(n+1) straight into
 * u_host, with nsteps > 1 one device-to-host copy brings the working copy back.  Any
 * other host memory: copied in, stepped, copied back.  Only the nx cells of each row
 * are guaranteed to be written back.  WCNS_ERR_ARG for a NULL pointer, nsteps < 0 or
 * a NaN dt/t_end; WCNS_ERR_NOMEM if the working copy cannot be allocated (first call). */
wcns_status wcns_step_host(wcns_ctx* ctx, void* u_host, double dt, int32_t nsteps, double t_end);

/* Device time control.  wcns_get_time synchronises the stream and returns the
 * device time and the number of steps that advanced it since the last set. */
wcns_status wcns_set_time(wcns_ctx* ctx, double t);
wcns_status wcns_get_time(wcns_ctx* ctx, double* t, int64_t* steps_taken);

/* Reductions over a grid buffer, results in FP64 on the host (synchronises).
 *   WCNS_REDUCE_SUM:     out[v] = sum over cells of a[v]            (nvar values)
 *   WCNS_REDUCE_L1:      out[v] = mean over cells of |a[v] - b[v]|  (b NULL: |a|)
 *   WCNS_REDUCE_LINF:    out[v] = max over cells of |a[v] - b[v]|   (b NULL: |a|)
 *   WCNS_REDUCE_MAXWAVE: out[d] = max over cells of |u_d| + c       (ndim values)
 * Accumulation is FP64 for both element types. */
wcns_status wcns_reduce(wcns_ctx* ctx, const void* a, const void* b, int32_t what, double* out);

/* Weight statistics of App. A for one evaluation of L(u): counts, over every one-sided
 * interpolation (both sides of every interface and every field, in both sweeps), the
 * base weights (the Z weights, or the JS weights before the M map) and the final
 * weights (FE mapped and renormalised, kept by the PFE switch, or unchanged) in nbins
 * equal bins of [0, 1], bin = floor(w * nbins + 1e-6) clamped to [0, nbins - 1] (the
 * ideal weights and control values lie on the edges of 1e4 bins; the offset keeps a
 * weight that round-off leaves just below an edge in the edge's bin).
 * Interfaces per line: the n + 5 the Eq. 3 difference reads (WCNS family) or the n + 1
 * of the two-point difference (WENO family); periodic lines count their wrapped halo
 * interfaces again.  hist: device array of 6 * nbins uint64_t counters, index
 * (kind * 3 + k) * nbins + bin with kind 0 = base, 1 = final and k the weight index;
 * the call adds to it (the caller zeroes it).  1 <= nbins <= 2^20, else WCNS_ERR_ARG.
 * Asynchronous on the context's stream; u must not be written meanwhile. */
wcns_status wcns_weight_hist(wcns_ctx* ctx, const void* u, int32_t nbins, uint64_t* hist);

/* Sets the boundary faces of the context's grid (faces NULL: back to the grid's bc).
 * Faces apply to wcns_rhs, wcns_step, wcns_step_host and wcns_weight_hist, not to the
 * adjoint (WCNS_ERR_UNSUPPORTED while faces are set).  Errors: WCNS_ERR_ARG for an
 * unknown type, a face on a periodic direction or a y face of a 1D grid, or a used
 * state with rho <= 0 or p <= 0; WCNS_ERR_UNSUPPORTED for wall / state faces on scalar
 * advection.  Captured step graphs are dropped (rebuilt on the next wcns_step). */
wcns_status wcns_set_faces(wcns_ctx* ctx, const wcns_faces* faces);

/* Self-test of the library's bounded device waits (no counterpart in the paper: it checks
 * the failure path of the kernels' waits without a GPU fault).  One thread waits, as the
 * banded stage does, on a completion counter that nothing increments, then, as the
 * TMA-staged tiles do, on an mbarrier armed for 16 bytes that no copy delivers.  Both
 * waits must give up (each after about a second at most): gave_up[0] (counter) and
 * gave_up[1] (mbarrier), a host array of 2, receive 1 when they did.  Each sets the
 * sticky error bit, so the next wcns_sync_status returns WCNS_ERR_TIMEOUT (and clears
 * it); the context stays usable.  Synchronises the context stream.
 * Errors: WCNS_ERR_ARG (null pointer), WCNS_ERR_CUDA. */
wcns_status wcns_selftest_waits(wcns_ctx* ctx, int32_t* gave_up);

/* Chooses how the RK stages of a 2D Euler grid run (steps (a)-(e) and the stage update
 * of wcns_step; the scheme itself, Eq. 2-3 with the TVD-RK3 or Eq. 16 stages, is the
 * same either way, and so is every result, bit for bit).
 *   banded = 0 (the default): an x-sweep launch over the whole grid, which writes the
 *     partial stage into a state-sized buffer, then a y-sweep launch that completes it.
 *   banded = 1: each stage is one cooperative persistent launch over bands of rows --
 *     the x-direction interfaces of a band write its partial stage into one of four
 *     band-sized ring slots, and the band's y-direction interfaces complete the stage
 *     from it -- so the partial stage stays in L2 and each stage moves about its
 *     algorithmic DRAM bytes (read u and u^n once, write the stage once) instead of about
 *     twice that.  On GB300 the sweeps are bound by instruction issue, not by DRAM, and
 *     the persistent loop's per-tile synchronisation costs more than the traffic saves
 *     (2048^2: 0.30 ms against 0.22 ms per FP32 stage), hence not the default.  It
 *     applies to 2D Euler grids of the default scheme configuration (FE weights with
 *     the Table 2 rows at kappa = 0.5, xi >= 1e4, Z p = 1, renormalised, HLLC,
 *     characteristic) with more than four bands of rows (bands are whole 75-row y
 *     tiles, at least 150 rows, at most 64 bands), in single precision only on grids
 *     wide enough for the four-interface x tiles.  The first banded = 1 call allocates
 *     the ring (4 slots of 4 x band rows x pitch elements); make it before any stream
 *     capture.
 * Errors: WCNS_ERR_ARG (null context), WCNS_ERR_UNSUPPORTED (banded = 1 where it does
 * not apply), WCNS_ERR_NOMEM.  Captured step graphs are dropped (rebuilt on the next
 * wcns_step). */
wcns_status wcns_set_stage_form(wcns_ctx* ctx, int32_t banded);

/* The reductions of wcns_reduce (SUM, L1, LINF only) without a context and without
 * any device allocation.  The paper has no counterpart: this serves callers that
 * cannot call cudaMalloc where they need the reduction -- a loop that reserved all of
 * its device memory up front and must not stall the device, or code inside a
 * framework whose allocator owns the device memory -- and therefore cannot create a
 * wcns_ctx either.  Its scratch is one 64 KiB array in device memory that every GPU
 * loading the library holds until the process exits.
 *   grid:   layout of a and b: 1 <= nvar <= 4; ndim, dtype, reserved, nx, ny and pitch
 *           obey the layout rules of wcns_init (ndim = 1 with ny > 1 is ny independent
 *           lines, reduced over all of their cells); lo/hi/bc are ignored.  Any other
 *           descriptor, nvar > 4 included, returns WCNS_ERR_ARG.
 *   a, b:   device grid buffers (b may be NULL: |a|); 16-byte aligned.
 *   what:   WCNS_REDUCE_SUM, _L1 or _LINF (else WCNS_ERR_UNSUPPORTED).
 *   stream: cudaStream_t the work is enqueued on (NULL: default stream).
 *   out:    DEVICE buffer of nvar doubles owned by the caller; written asynchronously.
 * The first call in a CUDA context (with the device current) resolves the array's
 * device address (a CUDA runtime query) and caches it for that context; make that
 * first call before any stream capture.  A device reset, or another context made
 * current on the device, starts a new context, whose first call repeats the lookup.
 * All calls share the array and it keeps the last call's contents: each call clears
 * the counters it needs on its own stream.  Calls that overlap on the GPU (unordered
 * streams) race on the array and give wrong results.  Safe to call from several host
 * threads (the address cache is locked); their GPU work must still not overlap. */
wcns_status wcns_reduce_noalloc(const wcns_grid* grid, const void* a, const void* b, int32_t what,
                                void* stream, double* out);

/* Adjoint of one TVD-RK3 step of fixed size dt > 0 (a hand-written reverse sweep of
 * the whole step: projection, interpolation, flux, flux difference and the three RK3
 * stages; the paper has no adjoint): given the checkpoint u_n and the cotangent lam_np1 of
 * u_{n+1} = S(u_n), writes lam_n = (dS/du_n)^T lam_np1.  The stage states u1, u2 are
 * recomputed from u_n (they overwrite the context's stage scratch); the reverse
 * sweeps differentiate the interface flux exactly, including the FE map (Eq. 20),
 * the Z/JS weights (Eq. 11, 14-15), the characteristic projection and the Roe
 * average, and scatter into cells by gathering (no atomics).
 * Supported: WCNS_EULER (ndim 1 or 2), WCNS_FLUX_LLF_FROZEN (a smooth flux), weights
 * JS / Z / FE / PFE, characteristic 0 or 1, WCNS_RK3, WCNS_FAMILY_WCNS; otherwise
 * WCNS_ERR_UNSUPPORTED.
 * lam_np1 and lam_n may be the same buffer; u_n must not alias either (the same pointer
 * returns WCNS_ERR_ARG; a partial overlap is not detected).  The first
 * call allocates two cotangent buffers of the context (nvar*ny*pitch each).
 * Asynchronous. */
wcns_status wcns_adjoint_step(wcns_ctx* ctx, const void* u_n, double dt, const void* lam_np1,
                              void* lam_n);

/* wcns_adjoint_step with the step's two inner TVD-RK3 stage states supplied by the caller
 * (RK-stage checkpoints, e.g. written by wcns_step_stages during the forward pass)
 * instead of recomputed from u_n: the reverse sweeps run at u2, u1 and u_n exactly as
 * in wcns_adjoint_step, so both give the same lam_n bit for bit when u1, u2 are the
 * step's stages.  u_n, u1, u2: device grid buffers of the step, 16-byte aligned, not
 * aliasing lam_np1 or lam_n (the same pointer returns WCNS_ERR_ARG).  Same options,
 * errors and allocation as wcns_adjoint_step.
 * Asynchronous. */
wcns_status wcns_adjoint_step_stages(wcns_ctx* ctx, const void* u_n, const void* u1, const void* u2, double dt,
                                     const void* lam_np1, void* lam_n);

/* One TVD-RK3 step of fixed size dt > 0 on u in place, as wcns_step(ctx, u, dt, 1, 0),
 * that also writes its two inner stage states, u1 = u + dt L(u) and
 * u2 = 3/4 u + 1/4 (u1 + dt L(u1)), into the caller's u1_out and u2_out (device grid
 * buffers, 16-byte aligned, distinct from u and from each other) instead of the
 * context's stage scratch: the forward half of RK-stage checkpointing for
 * wcns_adjoint_step_stages.  The device time advances by dt.  Errors: WCNS_ERR_ARG
 * (pointers, aliasing, dt <= 0), WCNS_ERR_UNSUPPORTED (integrator WCNS_RK4).
 * Asynchronous. */
wcns_status wcns_step_stages(wcns_ctx* ctx, void* u, double dt, void* u1_out, void* u2_out);

/* The device reciprocal behind every double-precision division of the sweeps and the CFL
 * step computation: out[i] = 1 / x[i] by two steps of Newton's iteration for the
 * reciprocal from the reciprocal unit's approximation.  No counterpart in the paper: it
 * lets a caller check that arithmetic against IEEE division (it differs by at most a
 * couple of ulps).  x, out: device arrays of n doubles, 8-byte aligned, owned by the
 * caller; inputs normal, finite and nonzero.  Asynchronous on `stream` (NULL: default
 * stream).  WCNS_ERR_ARG for a NULL pointer with n > 0, misalignment or n < 0. */
wcns_status wcns_reciprocal_f64(const double* x, double* out, int64_t n, void* stream);

/* Synchronises the context stream and returns (then clears) the sticky device
 * error; *nonphysical_interfaces (may be NULL) receives the number of interfaces
 * whose interpolated states fell back to the cell states since the last call. */
wcns_status wcns_sync_status(wcns_ctx* ctx, int64_t* nonphysical_interfaces);

const char* wcns_status_string(wcns_status s);

/* Per-kernel timing for benchmarks (no counterpart in the paper).  While enabled,
 * every kernel the context launches is bracketed by CUDA events recorded on the
 * context stream, and wcns_step launches kernels directly instead of replaying its
 * captured graph.  Enabling (or disabling) discards unread records. */
wcns_status wcns_profile_enable(wcns_ctx* ctx, int32_t on);

/* Synchronises the stream and returns, per kernel kind, its name (48-byte slots in
 * `names`), launches and total milliseconds since the last read, then resets them.
 * max_entries must be >= 11 (the number of kinds); *n_entries receives that number. */
wcns_status wcns_profile_read(wcns_ctx* ctx, int32_t max_entries, char* names, int64_t* launches,
                              double* ms, int32_t* n_entries);

/* Releases the context and its scratch (synchronises its stream first). */
void wcns_destroy(wcns_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Batched 1D Euler problems (many independent uneven grids, one launch per stage).
 * Problem k occupies columns offsets[k] .. offsets[k] + n[k] - 1 of a concatenated
 * buffer with `nvar` = 3 planes of `total` elements each (plane stride `total`),
 * on the domain [lo, hi] with boundary `bc` on both ends.  Every problem takes its
 * own CFL step each RK3 step; work is scheduled over (problem, tile) items by
 * persistent kernels, and each RK3 step replays one captured CUDA graph.
 * ------------------------------------------------------------------------- */

/* Creates a batch context.  offsets/n are host arrays of nprob entries; problems must
 * not overlap and must lie inside [0, total).  Copies them; allocates the stage
 * states, per-problem dt and time, and the work list (sorted by size, largest first).
 * `tile` = 0 lets the autotuner pick the tile (cells per work item) and the number of
 * resident blocks per SM on the first wcns_batch_step; otherwise one of 123, 251, 507. */
wcns_status wcns_batch_init(const int64_t* offsets, const int64_t* n, int32_t nprob, int64_t total,
                            double lo, double hi, int32_t bc, const wcns_params* params,
                            int32_t dtype, int32_t tile, void* stream, wcns_batch** out);

/* nsteps TVD-RK3 steps of every problem, each with its own CFL step clipped at t_end
 * (t_end <= 0: unclipped).  u_concat: device buffer described at wcns_batch_init.
 * Asynchronous (graph replays on the batch stream). */
wcns_status wcns_batch_step(wcns_batch* b, void* u_concat, int32_t nsteps, double t_end);

/* Reports the autotuned (or fixed) tile and blocks per SM, and the number of
 * candidates the autotuner timed (0 if fixed). */
wcns_status wcns_batch_config(wcns_batch* b, int32_t* tile, int32_t* blocks_per_sm,
                              int32_t* candidates_timed);

/* Per-problem device times (host array of nprob doubles); synchronises. */
wcns_status wcns_batch_times(wcns_batch* b, double* t_host);

wcns_status wcns_batch_sync_status(wcns_batch* b, int64_t* nonphysical_interfaces);
void wcns_batch_destroy(wcns_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* WCNS_H_ */
