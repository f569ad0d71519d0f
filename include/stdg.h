/*
 * stdg.h - C ABI of the GB300 space-time DG-SEM library (libstdg.so).
 *
 * Method: the space-time discontinuous Galerkin spectral element method of
 * Versbach, Linders, Kloefkorn and Birken, "Theoretical and Practical Aspects
 * of Space-Time DG-SEM Implementations" (arXiv:2201.05800).  One time slab
 * (one temporal element, Sec. 4) carries s = N_tau temporal LGL nodes; its
 * nonlinear system is Eq. DG_vs_RK:DG, solved by Jacobian-free Newton-Krylov
 * (Newton + restarted GMRES, Sec. 6.3 "Nonlinear solvers and preconditioning").
 *
 * Problem (Eq. general with S = 0): d_t u + div F_c(u) = div F_v on a
 * uniform periodic Cartesian grid (Sec. 3.1), with
 *   STDG_ADVECTION  u_t + a . grad u = 0              (r = 1)
 *   STDG_EULER      Euler equations, Eqs. eulereq/defu (r = d + 2,
 *                   u = (rho, rho v_1..rho v_d, E))
 *   STDG_BURGERS    u_t + div(u^2/2 (1,..,1)) = 0      (r = 1)
 * and the Rusanov (local Lax-Friedrichs) flux of Eq. flux:llf on every face
 * (exact upwind for advection).  For the scalar equations a viscous flux
 * F_v = nu grad u may be added (viscosity > 0): the symmetric interior penalty
 * form with the numerical flux H_v^IP of Sec. 3.1, penalty eta (default
 * 10 N^2, the paper's UFL choice) over h_e = h_a on faces normal to e_a, LGL
 * quadrature on elements and faces.  Initial data are nodal values on the LGL
 * nodes (interpolation = the quadrature projection of Eq. ode).
 *
 * Discrete residual evaluated by the library (the reading that makes its
 * Jacobian exactly Eq. Jacobian_ST):
 *   R(U) = (D_tau^T M_tau (x) I) U - (B_tau (x) I) U* + dt/2 (M_tau (x) I) F(U),
 *   U* = (u_prev, 0, ..., 0, U^s)                        (Eq. upwind_flux),
 * with F = M^-1 L_h the spatial DG-SEM operator (Eqs. elementint, surfaceint,
 * ode).  The slab solution is R(U) = 0 and the new state u^{n+1} = U^s (Eq. un).
 *
 * Layouts (all arrays dense, FP64, C order):
 *   element index e = (ez*Ky + ey)*Kx + ex, spatial node (iz, iy, ix) with ix
 *   fastest, r components fastest of all.
 *   state (one time level): u[e][iz][iy][ix][c]          stdg_state_len values
 *   slab  (s time nodes):   U[e][m][iz][iy][ix][c]       stdg_slab_len values
 *   node coordinates:       X[e][iz][iy][ix][a]          stdg_state_len/r*d values
 *
 * Pointers: ptr_kind STDG_HOST means ordinary host memory (copied in and out
 * on the context's stream, synchronously); STDG_DEVICE means device memory of
 * the current CUDA device, read and written in stream order on the context's
 * stream (the call returns once the work is enqueued, except where a value
 * must come back to the host).  The library never keeps a caller pointer past
 * the call and never frees caller memory; it owns the device memory inside a
 * context, freed by stdg_destroy.
 *
 * Errors: every call returns a stdg_status; no call throws, exits or traps.
 * stdg_last_error(ctx) gives a message for the last failing call on ctx.
 * A context is used by one host thread at a time.
 */
#ifndef STDG_H
#define STDG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stdg_ctx stdg_ctx;

typedef enum {
  STDG_OK = 0,
  STDG_ERR_INVALID_ARG = 1,      /* a NULL pointer, a size or option out of range      */
  STDG_ERR_OOM = 2,              /* device allocation failed or over hbm_budget_bytes  */
  STDG_ERR_CUDA = 3,             /* a CUDA runtime call failed (message in last_error) */
  STDG_ERR_NOT_CONVERGED = 4,    /* Newton hit newton_maxit before its tolerance       */
  STDG_ERR_GMRES_BREAKDOWN = 5,  /* GMRES stagnated at gmres_maxit with no progress    */
  STDG_ERR_NAN = 6,              /* a residual norm was NaN or Inf                     */
  STDG_ERR_TIMEOUT = 7,          /* reserved: a bounded device wait ran out            */
  STDG_ERR_CANCELLED = 8,        /* reserved: request cancelled by the caller          */
  STDG_ERR_UNSUPPORTED = 9       /* valid but not compiled in (e.g. dim/N combination) */
} stdg_status;

enum { STDG_ADVECTION = 0, STDG_EULER = 1, STDG_BURGERS = 2 };
enum { STDG_FLUX_RUSANOV = 0 };             /* Eq. flux:llf; upwind for advection       */
/* precision of Jv and the GMRES basis; STDG_MIXED_BF16: as STDG_MIXED_FP32 with the volume
 * contractions of the exact Jv on the tensor cores (BF16 inputs, FP32 accumulation), built for
 * the 3D Euler N = 3, s = 3 shape with STDG_JV_EXACT (other configurations: invalid) */
enum { STDG_FP64 = 0, STDG_MIXED_FP32 = 1, STDG_MIXED_BF16 = 2 };
enum { STDG_JV_FD = 0, STDG_JV_EXACT = 1 }; /* finite-difference JFNK or forward mode    */
enum { STDG_HOST = 0, STDG_DEVICE = 1 };
/* GMRES preconditioning of J dU = -R.  STDG_PRECOND_TEMPORAL_MASS solves the
 * left-scaled system (M_tau^-1 (x) I) J dU = -(M_tau^-1 (x) I) R: the rows of
 * temporal node m are divided by the LGL weight omega_m (a diagonal scaling;
 * the inner tolerance gmres_rtol then refers to the scaled residual).
 * STDG_PRECOND_POINT_BLOCK solves J P^-1 y = -R, dU = P^-1 y (right
 * preconditioning, so gmres_rtol refers to the true linear residual) with the
 * block of J that couples the s temporal nodes of one spatial node I: the
 * temporal part (D_tau^T M_tau - e_s e_s^T) of Eq. Jacobian_ST plus
 * dt/2 M_tau times the diagonal of the spatial Jacobian at I, which for the
 * Rusanov flux (Eq. flux:llf) is -sum over the faces through I of
 * lambda / (h_a w_end) (wave speed derivative dropped); one s x s matrix per
 * spatial node, rebuilt at every Newton step.  It pays on small grids (2D
 * vortex, 8 x 8 quads, N = 4, s = 4: 141 -> 90 GMRES iterations per slab) but
 * hardly on the 64 x 64 grid (108 -> 103), where the default
 * STDG_PRECOND_TEMPORAL_MASS is cheaper.  The Newton test always uses the
 * unscaled ||R||_2. */
enum { STDG_PRECOND_NONE = 0, STDG_PRECOND_TEMPORAL_MASS = 1, STDG_PRECOND_POINT_BLOCK = 2 };

/* Initial Newton iterate U0 of a slab.  CONSTANT: U0 = 1 (x) u^n.  EXTRAPOLATE: after a
 * solved slab of the same context, the previous slab's temporal polynomial evaluated at the
 * new slab's nodes, U0_m = sum_j l_j(tau_m + 2) U_j^prev (Lagrange basis l_j on the LGL nodes:
 * the temporal factor of the space-time expansion of Eq. StCoeff continued past its slab, with
 * tau in [-1, 1] on each slab); it is kept only when its residual is
 * below that of the constant guess.  The Newton target stays max(rtol ||R(1 (x) u^n)||, atol)
 * in both cases, so the accuracy asked of a slab does not depend on this choice. */
enum { STDG_PREDICTOR_CONSTANT = 0, STDG_PREDICTOR_EXTRAPOLATE = 1 };

typedef struct {
  int dim;                  /* spatial dimension d, 1..3                                 */
  int cells[3];             /* elements per direction (entries beyond dim ignored), >= 1 */
  double lo[3], hi[3];      /* periodic box [lo, hi] per direction                       */
  int N;                    /* spatial degree, n = N+1 LGL nodes per direction, 1..7      */
  int s;                    /* temporal LGL nodes N_tau (= Lobatto IIIC stages), 2..5    */
  int equation;             /* STDG_ADVECTION | STDG_EULER | STDG_BURGERS                */
  double adv_vel[3];        /* advection velocity a                                      */
  double gamma;             /* ratio of specific heats (Euler)                           */
  int flux;                 /* STDG_FLUX_RUSANOV                                         */
  double dt;                /* slab length Delta t_n > 0                                 */
  int precision;            /* STDG_FP64 | STDG_MIXED_FP32 | STDG_MIXED_BF16             */
  int jv_mode;              /* STDG_JV_FD | STDG_JV_EXACT                                */
  double newton_rtol;       /* stop when ||R||_2 <= max(rtol ||R(U0)||_2, atol)          */
  double newton_atol;
  int newton_maxit;         /* >= 1                                                      */
  int gmres_m;              /* restart length, 1..31                                     */
  double gmres_rtol;        /* inner tolerance eta (relative to ||R||)                   */
  int gmres_maxit;          /* total inner iterations per Newton step, >= 1              */
  size_t hbm_budget_bytes;  /* 0 = unlimited; else create fails with STDG_ERR_OOM above  */
  int precond;              /* STDG_PRECOND_NONE | _TEMPORAL_MASS (default) | _POINT_BLOCK */
  double viscosity;         /* nu >= 0: adds nu Laplace(u) (advection and Burgers only)  */
  double penalty;           /* interior penalty eta; <= 0 means the paper's 10 N^2       */
  int predictor;            /* STDG_PREDICTOR_CONSTANT (default) | _EXTRAPOLATE          */
} stdg_config_desc;

typedef struct {
  int newton_its;           /* Newton steps taken                                        */
  int gmres_its;            /* GMRES iterations summed over the Newton steps             */
  int residual_evals;       /* FP64 residual evaluations                                 */
  int jv_evals;             /* Jacobian-vector products                                  */
  double res0;              /* ||R(1 (x) u^n)||_2, the constant guess's residual          */
  double res_final;         /* ||R(U)||_2 at exit                                        */
} stdg_slab_stats;

/* Fill *desc with defaults (1D advection, N=3, s=3, FP64, FD Jv, GMRES(30)). */
void stdg_config_default(stdg_config_desc* desc);

/* Create a context on the current CUDA device; cuda_stream is a cudaStream_t
 * (NULL = legacy default stream) on which all work of the context is ordered.
 * Allocates every device buffer the slab solve needs (state, slab, residual,
 * Krylov basis of gmres_m+1 vectors).  *out is NULL on failure. */
stdg_status stdg_create(const stdg_config_desc* desc, void* cuda_stream, stdg_ctx** out);
stdg_status stdg_destroy(stdg_ctx* ctx);

size_t stdg_state_len(const stdg_ctx* ctx);   /* K * n^d * r                              */
size_t stdg_slab_len(const stdg_ctx* ctx);    /* K * s * n^d * r                          */
size_t stdg_coord_len(const stdg_ctx* ctx);   /* K * n^d * d                              */
size_t stdg_device_bytes(const stdg_ctx* ctx);/* device memory owned by the context       */

/* Physical coordinates of every spatial node (LGL nodes mapped to each element). */
stdg_status stdg_node_coordinates(const stdg_ctx* ctx, double* X, int ptr_kind);

/* Set / get the current state u^n (one time level). */
stdg_status stdg_set_state(stdg_ctx* ctx, const double* u, int ptr_kind);
stdg_status stdg_get_state(const stdg_ctx* ctx, double* u, int ptr_kind);
/* Get the last solved slab U (all s time nodes). */
stdg_status stdg_get_slab(const stdg_ctx* ctx, double* U, int ptr_kind);

/* Solve the current slab and advance: u^n <- U^s, t <- t + dt.  Newton-Krylov
 * starts from U0 = 1 (x) u^n, or with STDG_PREDICTOR_EXTRAPOLATE and a slab
 * solved since the last stdg_set_state from the extrapolated previous slab when
 * its residual is smaller (the stopping target is relative to ||R(1 (x) u^n)||
 * either way).  stats may be NULL.  Returns STDG_ERR_NOT_CONVERGED (state still
 * advanced to the last iterate) or STDG_ERR_NAN (state kept). */
stdg_status stdg_advance_slab(stdg_ctx* ctx, stdg_slab_stats* stats);

/* R = R(U; u_prev) (slab residual above).  U, R: slab_len; u_prev: state_len. */
stdg_status stdg_residual(stdg_ctx* ctx, const double* U, const double* u_prev, double* R, int ptr_kind);

/* Jv = J(U) v with J = dR/dU (Eq. Jacobian_ST), by the context's jv_mode:
 * STDG_JV_FD: [R(U + eps v) - R(U)]/eps with the exact linear temporal part,
 *             eps = sqrt(machine eps) (1 + ||U||_2) / ||v||_2;
 * STDG_JV_EXACT: forward-mode derivative (exact up to rounding).
 * u_prev does not enter J; it is accepted for symmetry with stdg_residual. */
stdg_status stdg_jv(stdg_ctx* ctx, const double* U, const double* u_prev, const double* v, double* Jv, int ptr_kind);

/* ||x||_2 of a device or host vector of slab_len values (FP64 accumulation). */
stdg_status stdg_slab_norm(stdg_ctx* ctx, const double* x, int ptr_kind, double* out);

/* F(U) at every temporal node: the spatial DG-SEM operator M^-1 L_h (Eq. ode)
 * applied to each time level of the slab U (slab layout in and out). */
stdg_status stdg_spatial_operator(stdg_ctx* ctx, const double* U, double* F, int ptr_kind);

/* J(U) v in FP32 with forward-mode (exact) derivatives, the product the inner
 * Krylov solve of STDG_MIXED_FP32 with STDG_JV_EXACT uses (Eq. Jacobian_ST):
 * ((D_tau^T M_tau - e_s e_s^T) (x) I) v + dt/2 (M_tau (x) I) F'(U) v.  Device
 * pointers to slab_len floats each (slab layout; U, v 16-byte aligned for the
 * bulk-copy kernel of the 2D n = 5, s = 4 and 3D n = 4, s = 3 Euler shapes,
 * else the general kernel runs; a context created with STDG_MIXED_BF16 runs
 * the volume contractions of the 3D shape on the tensor cores, BF16 inputs and
 * FP32 accumulation).  Synchronises the context stream; returns
 * STDG_ERR_TIMEOUT if a kernel's bounded wait (staged tile or tensor-core
 * accumulators) ran out. */
stdg_status stdg_jv_fp32(stdg_ctx* ctx, const float* U, const float* v, float* Jv);

/* One finite-difference Jacobian-vector launch exactly as GMRES issues it
 * (device pointers only): Jv = ((D_tau^T M_tau - e_s e_s^T) (x) I) v
 * + dt/2 (M_tau (x) I) [F(U + eps v) - F0] / eps, with F0 = F(U) supplied by the
 * caller (stdg_spatial_operator) and eps > 0. */
stdg_status stdg_jv_fd_apply(stdg_ctx* ctx, const double* U, const double* F0, const double* v, double eps,
                             double* Jv);

/* The method-of-lines DG-SEM + Lobatto IIIC slab residual (the LoDG form of
 * Sec. 5, Eq. DG_vs_RK:RK) with the Butcher matrix A = 1/2 Dtilde^-1,
 * Dtilde = D_tau + M_tau^-1 e_1 e_1^T (Eq. SBP_to_RK), from the same F(U):
 *   form 0:  R = U - 1 (x) u_prev - dt (A (x) I) F(U)
 *   form 1:  R = ((dt A)^-1 (x) I)(U - 1 (x) u_prev) - F(U)   (the A^-1 form whose
 *            Jacobian is Eq. Jacobian_Ainv)
 * U, R: slab layout (slab_len values); u_prev: state layout.  Both vanish at
 * the solution of stdg_residual (equivalence of the two formulations): the
 * space-time residual equals -(dt/2)(M_tau (x) I) times the form-1 residual. */
stdg_status stdg_lodg_residual(stdg_ctx* ctx, const double* U, const double* u_prev, double* R, int form,
                               int ptr_kind);

/* z = (P(U)^-1 (x) I_r) v with the point-block matrices P_I of
 * STDG_PRECOND_POINT_BLOCK built from the slab U (U, v, z: slab_len values).
 * For linear advection P_I (x) I_r is exactly the block of Eq. Jacobian_ST
 * that couples the temporal nodes and components of spatial node I.  FP64;
 * the library allocates the P^-1 storage of the context on the first call. */
stdg_status stdg_precond_apply(stdg_ctx* ctx, const double* U, const double* v, double* z, int ptr_kind);

/* Kernel accounting inside the library, per class: 0 space-time residual /
 * F(U), 1 Jacobian-vector product, 2 Gram-Schmidt and other vector kernels of
 * GMRES, 3 other (slab copies, predictor), 4 point-block preconditioner (build
 * and apply).  Launches are always counted; when timing is enabled every
 * kernel launch is also bracketed by CUDA events on the context stream and its
 * device time summed (ms stays 0 while disabled). */
typedef struct {
  int launches[5];
  double ms[5];
} stdg_profile;
stdg_status stdg_profile_enable(stdg_ctx* ctx, int on);
/* Synchronises the context stream, returns the sums since the last reset. */
stdg_status stdg_profile_read(stdg_ctx* ctx, stdg_profile* out, int reset);

/* ||x||_2 of a device vector without allocating anything on the device.
 *
 * No counterpart in the paper: this is a service entry point for callers that
 * cannot allocate device memory (stdg_create allocates the Krylov basis and
 * scratch of a context), for instance a host whose device memory is held
 * entirely by its own pool allocator, or a latency-critical loop that must not
 * call cudaMalloc/cudaFree (cudaFree synchronises the device).  It computes
 * the same norm as stdg_slab_norm up to FP64 rounding (FP64 squares, per-block
 * partial sums and a fixed-order final sum, but with its own blocking and a
 * device square root, so the two may differ in the last bits) for any length
 * up to STDG_NORM_NOALLOC_MAX_LEN.
 *   x            device pointer to len doubles (may be NULL when len == 0)
 *   out          device pointer to one double, receives the norm
 *   cuda_stream  cudaStream_t the two kernels are enqueued on (NULL = default)
 * The per-block partial sums live in one static device array of 4096 doubles
 * (32 KB) that every device which loads the library holds until exit.  It is
 * shared by all calls on a device: calls that may overlap on the GPU (e.g. on
 * two streams) race on it and must be ordered by the caller.  Every slot a
 * call reads was written by the same call, so no clearing is needed.  The
 * first call on a device, with that device current, looks up the array's
 * device address (cudaGetSymbolAddress) and keeps it for the life of the
 * process; make that first call before any stream capture.  The kept address
 * is valid only in the device's primary context (the one the CUDA runtime
 * uses) and only until that device is reset: after a cudaDeviceReset, or with
 * a driver-API context of the caller's own made current, do not call this
 * function again in the same process.  An error left pending on the calling
 * thread by earlier CUDA work is not consumed: the call then launches nothing
 * and returns STDG_ERR_CUDA, leaving the error for its owner to read.
 * Returns STDG_ERR_INVALID_ARG for a NULL pointer or
 * len > STDG_NORM_NOALLOC_MAX_LEN (nothing is launched), STDG_ERR_CUDA when the
 * set-up or a launch fails, else STDG_OK once the work is enqueued.  Calls no
 * allocating routine. */
#define STDG_NORM_NOALLOC_MAX_LEN ((size_t)67108864) /* 4096 blocks x 16384 values */
stdg_status stdg_slab_norm_noalloc(const double* x, size_t len, double* out, void* cuda_stream);

/* ===================================================================== batch
 * Batched slab solves (no counterpart in the paper's software, which solves
 * one slab system at a time; Sec. 6.3 for the Newton-Krylov method itself).
 * A batch holds many independent slab problems ("slots") of one spatial
 * dimension and equation that may differ in grid, N, s, dt and tolerances.
 * All slots advance together: every tick is one fixed sequence of kernel
 * launches over all slots, with the whole Newton-GMRES state of every slot on
 * the device (no host synchronisation inside a tick).  Per slot:
 *   Newton on R(U) = 0 from U0 = 1 (x) u^n, FP64 residual and update
 *   (stop: ||R||_2 <= max(newton_rtol ||R(U0)||_2, newton_atol)), each step
 *   solving J dU = -R by flexible GMRES(gmres_m) (no restart; the step takes
 *   the iterate after at most gmres_m iterations or at gmres_rtol; at most
 *   newton_maxit x ceil(gmres_maxit / gmres_m) such steps, the GMRES-iteration
 *   budget of the single-slab solver), right-
 *   preconditioned, with FP32 Krylov vectors and exact (forward-mode) FP32
 *   Jacobian-vector products; then u^{n+1} = U^s.  Preconditioner: Euler with
 *   inst->precond == STDG_PRECOND_POINT_BLOCK: the point-block P above; Euler
 *   otherwise: the temporal-mass scaling diag(1 / omega_m) (the point block
 *   stalls FGMRES on high-degree slabs with s = 2);
 *   scalar equations on grids whose element counts are powers of two (and
 *   whose lines fit 4096 values): the global inverse of
 *   C (x) I - dt/2 M_tau (x) (A_x (+) A_y), A_a the periodic 1D operator of the
 *   interior penalty form plus an upwind face dissipation with the slot's
 *   wave-speed bound (|a| for advection, max |u0| for Burgers), applied
 *   exactly by fast diagonalisation (FFT over the elements and per-mode
 *   eigenvectors along each direction, an s x s solve per spatial mode; see
 *   stdg_fdm_symbol); other scalar slots: the same with the element-local
 *   operator (neighbours set to zero) in place of A_a.
 * A slot's result does not depend on the other slots (no reduction crosses
 * slots, all reductions have a fixed order): bitwise the same alone or in a
 * mix.  Slot memory comes from one device arena of hbm_budget_bytes
 * allocated at creation; stdg_batch_add fails with STDG_ERR_OOM when the arena
 * has no room (admission by memory).  One host thread at a time per batch. */
typedef struct stdg_batch stdg_batch;
typedef struct {
  int dim;                  /* 1 or 2                                                    */
  int equation;             /* STDG_ADVECTION (1D, 2D), STDG_BURGERS (2D), STDG_EULER (2D) */
  int max_slots;            /* capacity of the slot table, >= 1                          */
  size_t hbm_budget_bytes;  /* arena for slot vectors, > 0                               */
} stdg_batch_desc;

/* Create a batch on the current device; cuda_stream as in stdg_create. */
stdg_status stdg_batch_create(const stdg_batch_desc* desc, void* cuda_stream, stdg_batch** out);
stdg_status stdg_batch_destroy(stdg_batch* b);
/* Admit one slab problem with initial state u0 (state layout, stdg_state_len
 * values of the problem, host or device pointer).  inst->dim and
 * inst->equation must match the batch; inst->gmres_m (1..31),
 * newton_rtol/atol/maxit, gmres_rtol and gmres_maxit are used; precision,
 * jv_mode, precond (but for STDG_PRECOND_POINT_BLOCK on scalar equations) and
 * predictor (a slot solves one slab from 1 (x) u0) are ignored (see above).
 * *slot receives the slot id.
 * STDG_ERR_OOM: the arena (or the slot table) is full; nothing changed. */
stdg_status stdg_batch_add(stdg_batch* b, const stdg_config_desc* inst, const double* u0, int ptr_kind, int* slot);
/* Run `ticks` ticks (>= 1), then report in *working how many admitted slots
 * have not finished (may be NULL).  Finished slots keep their results until
 * stdg_batch_remove. */
stdg_status stdg_batch_step(stdg_batch* b, int ticks, int* working);
/* Tick until no slot is working or max_ticks ticks ran. */
stdg_status stdg_batch_run(stdg_batch* b, int max_ticks, int* working);
/* *done = 1 once the slot's solve ended; *status = its stdg_status
 * (STDG_OK, STDG_ERR_NOT_CONVERGED, STDG_ERR_NAN); stats may be NULL. */
stdg_status stdg_batch_query(stdg_batch* b, int slot, int* done, int* status, stdg_slab_stats* stats);
/* u^{n+1} of a finished slot (u0 before), state layout. */
stdg_status stdg_batch_get_state(stdg_batch* b, int slot, double* u, int ptr_kind);
/* The slot's last Newton iterate U (slab layout, slab_len values). */
stdg_status stdg_batch_get_slab(stdg_batch* b, int slot, double* U, int ptr_kind);
/* Release a slot (its arena memory becomes free for new admissions). */
stdg_status stdg_batch_remove(stdg_batch* b, int slot);
/* Device bytes a problem would take in the arena (0 if invalid). */
size_t stdg_batch_slot_bytes(const stdg_batch* b, const stdg_config_desc* inst);
size_t stdg_batch_free_bytes(const stdg_batch* b);
/* Scheduling knobs of a batch (defaults: 0, 16, 1, 0).
 * share_quantum > 0 enables size-aware sharing: a slot of L space-time DOF
 *   takes part only in every k-th tick, k = clamp(round(L / share_quantum), 1,
 *   share_max_stride), so that very large slots do not set the tick time of
 *   the small ones (a slot's result does not change; only when it advances).
 * use_graphs: each stdg_batch_step is replayed as one captured CUDA graph of
 *   its ticks (recaptured when the slot set or the tick count changes).
 * autotune: elements per CTA of the operator kernels chosen by timing the
 *   candidates on a virtual 4096-element grid of each (dim, equation, N, s)
 *   class (the first time the class is admitted), cached for the process so
 *   that every slot of a class gets the same tiles; otherwise the largest tile
 *   of at most 256 nodes within 96 KB of shared memory. */
stdg_status stdg_batch_configure(stdg_batch* b, double share_quantum, int share_max_stride, int use_graphs,
                                 int autotune);
/* Slots that finished (as of the last step/run) and are not removed yet:
 * writes up to cap ids to slots, returns how many there are.  Host-side, no
 * synchronisation. */
int stdg_batch_done_slots(const stdg_batch* b, int* slots, int cap);
const char* stdg_batch_last_error(const stdg_batch* b);

/* ==================================================================== server
 * Continuous batching of slab solves (no counterpart in the paper).  A worker
 * thread owns a batch (above) on the device that is current at creation and
 * its own CUDA stream.  Submitted requests queue in arrival order; between
 * groups of ticks_per_round ticks the worker admits queued requests while the
 * arena (hbm_budget_bytes) and the slot table have room, so requests that
 * arrive while others run join their launches as memory frees up, and it
 * retires finished slots (result copied back, memory released).  A request
 * that alone exceeds the arena finishes with STDG_ERR_OOM.  A result is the
 * same as the batch would give for the request alone (see the batch section).
 * Submit and poll may be called from any host thread. */
typedef struct stdg_server stdg_server;
stdg_status stdg_server_create(const stdg_batch_desc* desc, int ticks_per_round, stdg_server** out);
/* Stops the worker (requests still queued or running are dropped). */
stdg_status stdg_server_destroy(stdg_server* s);
/* Queue one slab solve: inst as for stdg_batch_add, u0 = host initial state
 * (copied).  *ticket identifies the request. */
stdg_status stdg_server_submit(stdg_server* s, const stdg_config_desc* inst, const double* u0,
                               unsigned long long* ticket);
/* Wait up to wait_s seconds (0: do not wait) for the request.  *done = 1 once
 * it finished; then *status, *stats, the new state u (host, state length of
 * the request; may be NULL) and times[3] = {queue wait (submit -> admission),
 * service (admission -> done), latency (submit -> done)} in seconds (may be
 * NULL) are filled and the ticket is released. */
stdg_status stdg_server_poll(stdg_server* s, unsigned long long ticket, double wait_s, int* done, int* status,
                             stdg_slab_stats* stats, double* u, double* times);
/* Cancel a request.  A queued request is dropped; a running one releases its slot
 * before the worker's next round (the other slots are not affected).  The ticket
 * then reports done with STDG_ERR_CANCELLED; a request that already finished keeps
 * its result.  STDG_ERR_INVALID_ARG for an unknown (or already polled) ticket. */
stdg_status stdg_server_cancel(stdg_server* s, unsigned long long ticket);
/* Bound the submission queue: stdg_server_submit refuses a request with
 * STDG_ERR_OOM while max_queued requests wait for admission (0 = unbounded,
 * the default). */
stdg_status stdg_server_set_queue_limit(stdg_server* s, size_t max_queued);
/* The batch knobs of stdg_batch_configure, applied before the worker's next round. */
stdg_status stdg_server_configure(stdg_server* s, double share_quantum, int share_max_stride, int use_graphs,
                                  int autotune);
/* Admission policy, applied from the worker's next admission round.
 *   order 0: arrival order (the head of the queue blocks the ones behind it);
 *   order 1: the queued request with the fewest space-time DOF first (ties in
 *            arrival order): short requests do not wait behind long ones;
 *   max_running_dof > 0: no request is admitted while the admitted ones
 *            already hold that many space-time DOF (a larger request is
 *            admitted when nothing runs), so that each tick stays short;
 *            0: admission by device memory only.
 * Defaults: 0, 0.  A request's result does not depend on the policy (slots
 * are independent).  STDG_ERR_INVALID_ARG for an unknown order or a negative
 * or NaN cap. */
stdg_status stdg_server_set_policy(stdg_server* s, int order, double max_running_dof);
/* Counters since creation; returns the worker's fatal status (STDG_OK if none). */
stdg_status stdg_server_counters(stdg_server* s, unsigned long long* admitted, unsigned long long* completed,
                                 unsigned long long* ticks, int* queued, int* running, int* max_running);

const char* stdg_last_error(const stdg_ctx* ctx);
const char* stdg_status_string(stdg_status st);
/* Library version string. */
const char* stdg_version(void);
/* The LGL constants the CUDA path is built from (host only, no GPU needed): the
 * n-point Legendre-Gauss-Lobatto nodes x (ascending on [-1, 1]) and weights w
 * (Sec. 3.1; in time the same rule with n = s, Sec. 4) and the differentiation
 * matrix D[i*n + j] = l_j'(x_i) of the Lagrange basis on x (Eq. SBP).
 * 2 <= n <= 16; x, w: n doubles, D: n*n doubles, caller-owned. */
stdg_status stdg_lgl_constants(int n, double* x, double* w, double* D);
/* The matrix of STDG_PREDICTOR_EXTRAPOLATE (host only, no GPU needed):
 * E[m*s + j] = l_j(tau_m + 2) for the s-point temporal LGL rule, 2 <= s <= 5
 * (s*s doubles written to E, caller-owned).  STDG_ERR_INVALID_ARG otherwise. */
stdg_status stdg_predictor_matrix(int s, double* E);
/* Spectral data of the batch engine's global preconditioner (host only, no GPU
 * needed; no counterpart in the paper, which uses SOR on an assembled
 * Jacobian).  The periodic 1D operator A of K elements of width h (N+1 LGL
 * nodes): the symmetric interior penalty form of -nu d^2/dx^2 (Sec. 3.1, penalty
 * eta, eta <= 0 meaning 10 N^2, h_e = h) plus the upwind dissipation lam/2 [[u]]
 * of the Rusanov flux (Eq. flux:llf) with the constant speed lam.  Its
 * eigenvectors are phi[e][i] = exp(2 pi i k e / K) V_k[i][j], k < K, j <= N:
 * lambda[k (N+1) + j] receives the eigenvalue, Vre / Vim[(k (N+1) + i)(N+1) + j]
 * the real and imaginary parts of V_k[i][j] (caller-owned arrays of K (N+1) and
 * K (N+1)^2 doubles).  STDG_ERR_INVALID_ARG for N outside 1..7, K < 1, h <= 0,
 * nu < 0, lam < 0 or a NULL pointer; STDG_ERR_NOT_CONVERGED if an eigensolve
 * did not converge. */
stdg_status stdg_fdm_symbol(int N, int K, double h, double nu, double eta, double lam, double* lambda,
                            double* Vre, double* Vim);

#ifdef __cplusplus
}
#endif
#endif /* STDG_H */
