/*
 * liblbm: GB300 (sm_103a) implementation of one time step of the double
 * multiple-relaxation-time lattice Boltzmann model for solid-liquid phase
 * change with natural convection in porous media at the REV scale
 * (Liu & He, arXiv:1503.08406).
 *
 * One step advances two coupled lattices and the liquid fraction:
 *   - D2Q9 MRT flow lattice with the generalized non-Darcy body force,
 *     Eq. (4)-(6), (13)-(29), on liquid nodes, halfway bounce-back on links
 *     into solid or wall nodes;
 *   - D2Q5 MRT temperature lattice with the latent-heat source, Eq. (30)-(39),
 *     non-equilibrium extrapolation on thermal wall nodes (Sec. 4 preamble);
 *   - the iterative enthalpy method for the liquid fraction, Eq. (40)-(42)
 *     with the inner iteration of Sec. 3.2.
 *
 * Conventions (all entry points):
 *   - fields are row-major [ny][nx] float32 arrays, x fastest;
 *   - the caller owns every pointer it passes; the library copies from or
 *     into it during the call (or, for device pointers, on the context's
 *     stream) and never keeps it;
 *   - the context owns its device state (populations, liquid fraction,
 *     material fields, scratch), either in memory it allocated itself or in
 *     a caller-provided workspace (see lbm_create);
 *   - every int-returning call returns LBM_OK (0) or a negative LBM_ERR_*;
 *     nothing aborts, throws or exits across this boundary;
 *   - work is queued on the stream given to lbm_create; calls that return
 *     host data synchronise that stream.
 */
#ifndef LBM_H
#define LBM_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_ERR_INVALID_ARG (-1)  /* bad size, bad parameter, NULL where data is needed */
#define LBM_ERR_CUDA (-2)         /* a CUDA call failed; the context may be unusable */
#define LBM_ERR_NONFINITE (-3)    /* a reduction found NaN or Inf in the state */
#define LBM_ERR_NOT_CONVERGED (-4)/* an inner enthalpy iteration hit max_inner_iters */
#define LBM_ERR_OOM (-5)          /* allocation failed or workspace too small */
#define LBM_ERR_NO_DEVICE (-6)    /* no usable sm_103a device */
#define LBM_ERR_TIMEOUT (-7)      /* a bounded device-side wait gave up (a bulk copy into shared
                                     memory did not arrive); the results of that step are invalid */

/* Boundary condition of one side. Periodic sides come in pairs (left/right,
 * bottom/top). A non-periodic side's outer row or column is a wall node:
 * no flow, fixed liquid fraction, halfway bounce-back for the flow lattice,
 * non-equilibrium extrapolation for the temperature lattice (Sec. 4). */
enum { LBM_BC_PERIODIC = 0, LBM_BC_DIRICHLET = 1, LBM_BC_ADIABATIC = 2 };

/* Storage of the populations in device memory (lbm_params.storage).  All
 * arithmetic is FP32 in every case; f_l, phi and K are always FP32.  The
 * 16-bit forms store f_i - w_i rho0 and g_i - w~_i T_m (T_m = (T_s + T_l)/2,
 * where the phase change needs the finest resolution of T); they cut
 * the stream-collide traffic from 124 to 68 bytes per flow node at the cost of
 * that rounding every step (the error against the oracle is measured, not
 * bounded). */
enum { LBM_STORAGE_FP32 = 0, LBM_STORAGE_FP16 = 1, LBM_STORAGE_BF16 = 2 };
enum { LBM_SIDE_LEFT = 0, LBM_SIDE_RIGHT = 1, LBM_SIDE_BOTTOM = 2, LBM_SIDE_TOP = 3 };

/* Inputs. Dimensionless groups as in Eq. (9). A negative tau_nu, tau_T or
 * g_beta is derived (Sec. 4.3): tau_nu = 1/2 + Ma J H sqrt(3 Pr)/sqrt(Ra),
 * tau_T = 1/2 + lambda c_s^2 (tau_nu - 1/2)/(J sigma c_sT^2 Pr),
 * g_beta = Ra nu_l alpha_l/(dT H^3). Zero relaxation rates take the Sec. 4
 * values s_e = s_eps = 1.1, s_q = 1.2, zeta_e = zeta_nu = 1.5. Zero H means
 * H = ny; zero dT, rho0, J or lambda_ mean 1. With flow = 0 (vartheta = 0,
 * pure conduction) tau_T must be given. */
typedef struct {
  int32_t nx, ny;                 /* lattice nodes, >= 3 each */
  int32_t bc[4];                  /* LBM_BC_* for left, right, bottom, top */
  double  T_bc[4];                /* Dirichlet wall temperatures, same order */
  int32_t flow;                   /* 1: flow lattice on (vartheta = 1); 0: conduction */
  double  Ra, Pr, Ma, J, lambda_, sigma, St, dT, H;
  double  T_ref;                  /* T_0 of the Boussinesq term, Eq. (5) */
  double  T_s, T_l;               /* solidus, liquidus, Eq. (41)-(42); T_s == T_l allowed */
  double  varpi;                  /* D2Q5 parameter, -4 < varpi < 1 (paper: -2) */
  double  rho0;
  double  tau_nu, tau_T, g_beta;
  double  s_e, s_eps, s_q, zeta_e, zeta_nu;
  double  f_act;                  /* a node carries flow when f_l >= f_act (default 1e-3) */
  int32_t max_inner_iters;        /* cap of one inner enthalpy solve (default 1000) */
  double  inner_tol;              /* inner iteration stop: max |f(k+1) - f(k)| (FP32 path: >= 1e-6) */
  double  screen_tol;             /* phase-change screen margin in temperature: 0 = 1e-7 of the
                                     temperature scale; < 0 = no screen, every tile is solved */
  int32_t kernel_variant;         /* stream-collide kernel: 0 auto (TMA-staged where the lattice
                                     qualifies), 1 ordinary loads, 2 TMA-staged (falls back to 1
                                     where the lattice does not qualify); results are identical */
  int32_t storage;                /* LBM_STORAGE_*: population storage (default FP32) */
  double  alpha_ratio;            /* alpha_l / alpha_s (Sec. 4.1): tau_T (the liquid value) is
                                     applied per node as 1/2 + (tau_T - 1/2)(f_l + (1 - f_l)/ratio),
                                     i.e. alpha_e = alpha_l f_l + alpha_s (1 - f_l); 0 or 1: one
                                     diffusivity for both phases */
  int32_t check_every;            /* > 0: lbm_step scans every population and f_l for NaN or
                                     Inf after every check_every steps (one read of the state,
                                     queued on the stream); lbm_status then reports
                                     LBM_ERR_NONFINITE.  0: no sentinel */
  double  sigma_solid;            /* heat-capacity ratio of the solid, Eq. (7): > 0 and != sigma
                                     makes sigma linear in f_l, sigma_solid + f_l (sigma -
                                     sigma_solid), taken at f_l(n) per node in tau_T (the given
                                     tau_T belongs to the liquid), in n^eq of Eq. (34), in the
                                     wall extrapolation and in the latent coefficient
                                     a = phi dT / (sigma St) of Eq. (38); 0: one sigma */
  int32_t flow_walls;             /* 1: flow walls by non-equilibrium extrapolation (Sec. 4):
                                     a wall node whose inward node (the diagonal one at a
                                     corner) carries flow takes f^eq(rho_f, 0) + f(x_f) -
                                     f^eq(rho_f, u_f) before collision, collides with x_f's
                                     T, f_l, phi and K and streams like a flow node, and links
                                     into it stream; 0: links into wall nodes reflect halfway.
                                     Ignored without the flow lattice; the coupled adjoint
                                     refuses it */
  int32_t flow_front;             /* 1: no-slip on the moving solid-liquid interface by the
                                     same extrapolation (Sec. 4): a link from a flow node x
                                     into a lattice node without flow returns, in place of x's
                                     reflected population, the one that node would stream
                                     back as a boundary node extrapolated from x
                                     (f^eq(rho_x, 0) + f(x) - f^eq(rho_x, u_x) collided with
                                     x's T, f_l, phi and K); 0: halfway bounce-back.  Links
                                     into wall nodes follow flow_walls.  Ignored without the
                                     flow lattice; the coupled adjoint refuses it */
} lbm_params;

typedef struct lbm_ctx lbm_ctx;

/* Bytes of device workspace a context with these parameters needs; lets a
 * caller (e.g. a framework's caching allocator) provide the memory itself. */
int lbm_workspace_bytes(const lbm_params* p, size_t* bytes);

/* Validate p, derive the lattice parameters and set up device state on the
 * current CUDA device. `stream` is a cudaStream_t (NULL: the legacy default
 * stream); all device work of the context is queued on it. `workspace` is a
 * device pointer of at least lbm_workspace_bytes() bytes, 256-byte aligned,
 * that the context uses for all its device state and keeps using until
 * lbm_destroy; the caller keeps ownership and must not free it before then.
 * Pass NULL to have the library allocate (and later free) the memory.
 * On error *out is NULL. */
int lbm_create(const lbm_params* p, void* stream, void* workspace, size_t workspace_bytes,
               lbm_ctx** out);

/* Release the context (and the memory the library allocated). NULL is a no-op. */
void lbm_destroy(lbm_ctx* c);

/* Derived lattice quantities: tau_nu, tau_T, nu_e, nu_l, alpha_e, g_beta,
 * c_sT^2, latent coefficient dT/(sigma St). */
int lbm_derived(const lbm_ctx* c, double out[8]);

/* Load the material and initial fields (nx*ny floats each) and reset the
 * populations to the rest equilibria f = f^eq(rho0, 0), Eq. (29), and
 * g = g^eq(T0, 0), Eq. (39). phi: porosity in (0,1] (flow needs < 1);
 * K: fully liquid permeability in lattice units, > 0, +inf = no porous drag;
 * T0: initial temperature; fl0: initial liquid fraction in [0,1] (kept fixed
 * on wall nodes). wall_T_left: NULL or ny floats replacing T_bc[LEFT] row by
 * row on a Dirichlet left wall. device_ptrs != 0: the pointers are device
 * memory (copies are queued on the context stream); 0: host memory (the call
 * synchronises). Validation of host inputs returns LBM_ERR_INVALID_ARG. */
int lbm_set_fields(lbm_ctx* c, const float* phi, const float* K, const float* T0,
                   const float* fl0, const float* wall_T_left, int device_ptrs);

/* Queue nsteps >= 0 time steps on the context stream. Returns launch and
 * argument errors only; device-side conditions (an inner iteration that hit
 * its cap, a non-finite value found by the sentinel, a wait that gave up) are
 * reported by lbm_status.  Steps are replayed from CUDA graphs of up to 64
 * steps, keyed by the step parity they start at and their length; a graph is
 * captured the first time it is needed (host work before its launch). */
int lbm_step(lbm_ctx* c, int64_t nsteps);

/* Capture, without running anything, the CUDA graphs that lbm_step(c, nsteps)
 * called now would use, so that the call itself only launches them.  No-op
 * while timing is on.  LBM_ERR_CUDA if a capture fails. */
int lbm_prepare(lbm_ctx* c, int64_t nsteps);

/* Synchronise the stream and report deferred device-side conditions, in this
 * order: LBM_ERR_NONFINITE if the sentinel (lbm_params.check_every) found NaN
 * or Inf in the state (kept until lbm_set_fields or lbm_set_state);
 * LBM_ERR_TIMEOUT if a bounded device-side wait gave up (the flag is then
 * cleared); LBM_ERR_NOT_CONVERGED if any inner enthalpy iteration hit
 * max_inner_iters since the last call (the flag is then cleared); else LBM_OK. */
int lbm_status(lbm_ctx* c);

/* Self-check of the device-side timeout path: queue one CTA that waits, with
 * the same bounded wait the stream-collide kernel uses for its bulk copies, on
 * a shared-memory barrier that nothing ever completes, giving up after
 * limit_ns nanoseconds (1e3 <= limit_ns <= 1e9).  When it gives up it sets the
 * flag a timed-out copy sets, so the next lbm_status returns LBM_ERR_TIMEOUT.
 * The context's state is not touched.  LBM_ERR_INVALID_ARG outside the range. */
int lbm_check_wait(lbm_ctx* c, int64_t limit_ns);

/* Steps taken since the last lbm_set_fields / lbm_set_state. */
int64_t lbm_steps_done(const lbm_ctx* c);

/* Kernels lbm_step has launched on this context (directly or in CUDA graphs),
 * for accounting: a step is 3 kernels (fused, enthalpy solve, enthalpy commit);
 * inside a graph the fused pass of every step but the first is split in two
 * (tiles away from the front, run concurrently with the previous step's
 * enthalpy kernels, and tiles near it). */
int64_t lbm_kernel_launches(const lbm_ctx* c);

/* Stream-collide kernel this context runs: 1 ordinary loads, 2 TMA-staged
 * kernel (lattices walled on all four sides whose rows are a multiple of 16
 * bytes, i.e. nx a multiple of 4 (FP32) or 8 (16-bit storage), nx >= 40
 * (48 with 16-bit storage), ny >= 10); -1 for NULL. */
int lbm_kernel_variant(const lbm_ctx* c);

/* Autotuner: times `trial_steps` (even, >= 2) graph-replayed
 * steps of this context for each stream-collide configuration -- the ordinary-
 * load kernel and, where the lattice qualifies, the TMA-staged kernel with
 * 2, 3, 4, 5, 6 or 8 tiles of 32x8 nodes per CTA -- and keeps the fastest.
 * Every configuration computes the same step (bit for bit), so the trial steps
 * are real steps of the run: the context advances by 2 trial_steps per
 * configuration (one untimed run that captures the graphs, one timed), plus
 * one step first if its step count is odd.  Synchronises.  *variant and *tiles_per_cta (either may be
 * NULL) receive the choice (tiles_per_cta 0 for the ordinary-load kernel). */
int lbm_autotune(lbm_ctx* c, int trial_steps, int32_t* variant, int32_t* tiles_per_cta);

/* Adjoint of the conduction step.  Runs nsteps steps forward from the
 * context's current state and returns the melted fraction J (mean f_l over
 * non-wall nodes) after them, with its gradient with respect to the porosity
 * field (d_phi, nx*ny) and to the left wall's temperature profile
 * (d_wall_T_left, ny), by the discrete adjoint of the step (the reverse of the
 * wall extrapolation, collision, streaming, latent source and, by the implicit
 * function theorem, the enthalpy fixed point; the clamp of Eq. (42)
 * differentiates to 1 on the nodes with 0 < f_l < 1 after the step, else 0).
 * The reverse sweep needs f_l after every step.  checkpoint_every = 0: kept
 * for all steps (4 bytes per node and step) when that takes at most half the
 * free device memory, else as for sqrt(nsteps); checkpoint_every = K > 0: the
 * whole state kept every K steps and the steps between recomputed (a CUDA
 * graph per segment).  All choices give the same result.  Jacobi sweeps solve
 * the fixed point's adjoint per step until the largest change is within 4e-7
 * of the value, at most mu_sweeps (0: 64).  The context ends where the forward
 * run left it (nsteps further on).  Covers: no flow (flow = 0), periodic in y
 * with wall columns at x = 0 (Dirichlet, the profile) and x = nx - 1
 * (Dirichlet or adiabatic), FP32 storage, one thermal diffusivity;
 * LBM_ERR_INVALID_ARG otherwise.  Allocates its buffers with cudaMalloc
 * (LBM_ERR_OOM if that fails) and synchronises.  device_ptrs: d_phi and
 * d_wall_T_left are device (1) or host (0) pointers. */
int lbm_adjoint_melt(lbm_ctx* c, int64_t nsteps, int32_t checkpoint_every, int32_t mu_sweeps,
                     float* d_phi, float* d_wall_T_left, double* J, int device_ptrs);

/* Device time (CUDA events on the context stream, ms) of the last adjoint call
 * on this context (lbm_adjoint, lbm_adjoint_melt or lbm_adjoint_coupled):
 * ms[0] its forward run with the saves it makes, ms[1] its reverse sweep
 * (recomputation of checkpointed segments included); zeros before the first. */
int lbm_adjoint_timing(const lbm_ctx* c, double ms[2]);

/* Objectives of lbm_adjoint. */
enum { LBM_OBJ_MELT = 0, LBM_OBJ_NUSSELT = 1 };

/* lbm_adjoint_melt for a chosen objective: LBM_OBJ_MELT as there;
 * LBM_OBJ_NUSSELT: the left-wall Nusselt number (lbm_reduce's out[3]: the
 * second-order one-sided gradient -(-3 T_w + 4 T_1 - T_2)/2 times H/dT,
 * averaged over the rows) after each of the nsteps steps, averaged over them;
 * its gradient has a direct term in the wall profile.  The Nusselt objective
 * needs nx >= 5.  Everything else as for lbm_adjoint_melt. */
int lbm_adjoint(lbm_ctx* c, int objective, int64_t nsteps, int32_t checkpoint_every,
                int32_t mu_sweeps, float* d_phi, float* d_wall_T_left, double* J,
                int device_ptrs);

/* Adjoint of the coupled step (flow lattice on or off).  Runs nsteps steps forward
 * from the context's current state and returns the objective J (LBM_OBJ_MELT
 * or LBM_OBJ_NUSSELT, as for lbm_adjoint) with its gradients with respect to
 * the porosity field (d_phi, nx*ny), the logarithm of the permeability field
 * (d_lnK, nx*ny) and the left wall's temperature profile (d_wall_T_left, ny):
 * the discrete adjoint of the flow collision with the Darcy-Forchheimer force
 * and buoyancy (Eq. (4)-(6), (16)-(28)), of streaming with bounce-back (the
 * flow mask f_l(n) >= f_act held fixed), of the thermal step with the
 * velocity (Eq. (34)-(36), the wall extrapolation of Sec. 4) and of the
 * enthalpy fixed point (Eq. (38)-(42)).  The reverse sweep needs the state of
 * every step (f, g and f_l: 60 bytes per node).  checkpoint_every = 0: every
 * state kept when that takes at most half the free device memory, else as
 * for sqrt(nsteps); checkpoint_every = K > 0: the whole state kept every K
 * steps, and each segment recomputed from its checkpoint and reversed from
 * one CUDA graph replay (the forward run replays graphs too).  All choices
 * give the same result bit for bit.  LBM_ERR_OOM when the kept states would
 * exceed the free memory.  Covers: FP32 storage, one heat-capacity ratio,
 * the flow lattice on or off, one thermal diffusivity or alpha_l != alpha_s
 * (alpha_ratio, Sec. 4.1), a Dirichlet left wall (walls left and right,
 * nx >= 5), halfway bounce-back on walls and front (flow_walls = flow_front =
 * 0), no timing; LBM_ERR_INVALID_ARG otherwise.  The context ends where the
 * forward run left it.  Allocates its buffers with cudaMalloc and
 * synchronises.  device_ptrs: the three gradient
 * arrays are device (1) or host (0) pointers. */
int lbm_adjoint_coupled(lbm_ctx* c, int objective, int64_t nsteps, int32_t checkpoint_every,
                        int32_t mu_sweeps, float* d_phi, float* d_lnK, float* d_wall_T_left,
                        double* J, int device_ptrs);

/* Batches.  A batch advances several contexts together: each
 * lbm_batch_step replays one CUDA graph holding LBM_BATCH_STEPS steps of every
 * context, each context's kernels on its own branch, so small lattices fill the
 * GPU together instead of one after another.  The contexts stay owned by the
 * caller, must outlive the batch, and must have the same step count modulo 2
 * when lbm_batch_step is called; each keeps its own parameters, size and
 * kernel configuration (tune them before lbm_batch_create).  The results of
 * every context are bit for bit those of stepping it alone. */
#define LBM_BATCH_STEPS 32
typedef struct lbm_batch lbm_batch;
/* stream: where lbm_batch_step launches (NULL: the default stream).  The graph
 * is captured on the first lbm_batch_step.  LBM_ERR_INVALID_ARG for count < 1,
 * NULL or repeated contexts. */
int lbm_batch_create(lbm_ctx* const* ctxs, int count, void* stream, lbm_batch** out);
/* Advance every context by nsteps (>= 0): whole graphs of LBM_BATCH_STEPS
 * steps, the rest through each context's own lbm_step.  Ordered after work
 * already queued on each context's stream, and before work queued there later.
 * Asynchronous; LBM_ERR_INVALID_ARG if a context has timing enabled or the
 * contexts' step counts differ in parity. */
int lbm_batch_step(lbm_batch* b, int64_t nsteps);
/* How the batch graph launches its kernels: 1 when every context runs the
 * TMA-staged stream-collide kernel on FP32 storage with the same flow setting,
 * no flow walls, and there are at most 64 contexts: each pass of a step (far
 * and near stream-collide tiles, enthalpy solve, commit) is then one launch
 * over all contexts, each context on its own range of CTAs; 0 otherwise: one
 * graph branch per context.  The results are the same bits either way. */
int lbm_batch_mode(const lbm_batch* b);
void lbm_batch_destroy(lbm_batch* b);

/* Macroscopic fields at the current time (each nx*ny floats, NULL to skip):
 * velocity from Eq. (26)-(28) (zero on nodes without flow), rho from
 * Eq. (24), T from Eq. (33) (wall nodes: the temperature the wall imposes),
 * and f_l. device_ptrs as in lbm_set_fields; host outputs synchronise. */
int lbm_get_macros(lbm_ctx* c, float* ux, float* uy, float* rho, float* T, float* fl,
                   int device_ptrs);

/* FP64 sums over non-wall nodes: out[0] total mass sum f_i, out[1] total
 * enthalpy sum (T + a f_l) with a = phi dT/(sigma St) (Eq. 38), out[2] mean
 * f_l, out[3] mean Nusselt number on the left wall (second-order one-sided
 * gradient times H/dT). Synchronises. LBM_ERR_NONFINITE if a sum is not finite. */
int lbm_reduce(lbm_ctx* c, double out[4]);

/* Checkpoint: populations in natural layout, f[9][ny][nx] as deviations
 * f_i - w_i rho0 from the rest equilibrium (the stored form), g[5][ny][nx],
 * and f_l[ny][nx] (NULL to skip). lbm_set_state restores them and resets the
 * step parity, so a state saved and restored continues bit for bit. */
int lbm_get_state(lbm_ctx* c, float* f, float* g, float* fl, int device_ptrs);
int lbm_set_state(lbm_ctx* c, const float* f, const float* g, const float* fl, int device_ptrs);

/* Per-kernel timing with CUDA events on the context stream. enable != 0
 * starts recording (and clears earlier records and counters); while it is on,
 * lbm_step launches kernel by kernel (no CUDA graph, no overlap) with events
 * between the kernels. lbm_timing_read synchronises and returns in ms[0..3]
 * the summed milliseconds, over the recorded steps, of the fused
 * stream-collide kernel, of a preparation stage (zero in this version; kept
 * for layout), of the enthalpy solve kernel and of the enthalpy commit
 * kernel; also the number of
 * steps timed, the number of enthalpy tiles solved and the largest number of
 * inner sweeps one tile needed (NULL counters are skipped). */
int lbm_timing(lbm_ctx* c, int enable);
int lbm_timing_read(lbm_ctx* c, double ms[4], int64_t* steps_timed, int64_t* tiles_solved,
                    int32_t* max_sweeps);

/* Kernel trace, for finding where a step's time goes (graph replays run
 * kernels side by side, which per-kernel timing cannot show).  capacity > 0:
 * allocate a device buffer of that many records (cudaMalloc; LBM_ERR_OOM if
 * it fails), empty it and start recording; 0: stop and free it.  While on,
 * every CTA of the TMA-staged stream-collide kernel and of the enthalpy solve
 * and commit kernels appends one record when it ends: kind (100 x step parity
 * + 10 + pass for the stream-collide kernel, pass 0 all tiles, 1 tiles away
 * from the front, 2 tiles near it; + 20 the solve; + 30 the commit), the step
 * stamp (the same for all launches of one step), and the CTA's start and end
 * times in ns of the GPU's global timer.  Records beyond the capacity are
 * dropped.  Synchronises; CUDA graphs are captured again afterwards. */
int lbm_trace(lbm_ctx* c, int64_t capacity);
/* Copy up to max_records records (4 int64 each, in the order CTAs ended) to
 * host memory, set *count, and empty the buffer.  Synchronises. */
int lbm_trace_read(lbm_ctx* c, int64_t* records, int64_t max_records, int64_t* count);

/* Largest lattice height (rows) lbm_reduce_state_noalloc accepts. */
#define LBM_NOALLOC_MAX_ROWS 16384

/* The sums of lbm_reduce, computed from a checkpoint the caller holds, without
 * allocating any memory. The paper has no counterpart: this is an operational
 * entry point for callers that cannot allocate device memory, e.g. a framework
 * whose caching allocator owns all device memory and forbids side allocations,
 * or monitoring code that runs inside a fixed memory budget and must not take
 * device memory from the job it watches. Unlike lbm_create, it needs no
 * context and no workspace.
 * Inputs (device pointers, natural layout, FP32, as lbm_get_state writes them
 * for every population storage; p->storage is ignored): f[9][ny][nx] as
 * deviations f_i - w_i rho0, g[5][ny][nx], fl and phi [ny][nx]; wall_T_left:
 * NULL or ny device floats (the left-wall profile the context was given).
 * p supplies nx, ny, bc, T_bc, sigma, St, dT, H, rho0.
 * out (host, 4 doubles): total mass, total enthalpy, mean f_l, mean left-wall
 * Nusselt number, as lbm_reduce defines them.
 * The call is synchronous: it queues its kernels on `stream` (a cudaStream_t;
 * NULL: legacy default stream), copies the sums to host memory and synchronises
 * that stream before it returns. Scratch is a fixed array of
 * LBM_NOALLOC_MAX_ROWS x 6 doubles (768 KB) in the library's device memory,
 * which every GPU that loads the library keeps until the process exits;
 * ny > LBM_NOALLOC_MAX_ROWS returns LBM_ERR_INVALID_ARG. The first call on a
 * device looks up the array's device address (with that device current), so
 * make that first call before any stream capture.
 * All calls share the array: calls whose kernels may overlap on the GPU (on
 * different streams without ordering) race and can return wrong sums.
 * Returns LBM_OK, LBM_ERR_INVALID_ARG, LBM_ERR_CUDA, LBM_ERR_NO_DEVICE or
 * LBM_ERR_NONFINITE (a sum is not finite; out is still written). */
int lbm_reduce_state_noalloc(const lbm_params* p, const float* f, const float* g, const float* fl,
                             const float* phi, const float* wall_T_left, void* stream,
                             double out[4]);

/* Static text for an LBM_* code. */
const char* lbm_error_string(int code);

#ifdef __cplusplus
}
#endif
#endif
