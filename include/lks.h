/*
 * lks.h -- C ABI of the GB300 (sm_103a) implementation of the Lattice Kinetic
 * Scheme (LKS) state march, the Adjoint Lattice Kinetic Scheme (ALKS) and the
 * design sensitivity of Tanabe, Yaji and Ushijima, "Adjoint lattice kinetic scheme
 * for topology optimization in fluid problems" (arXiv 2411.03090).
 *
 * The calls follow the paper's optimization procedure (Sec. 2.7):
 *   Step 2  state fields by LKS               -> lks_forward
 *   Step 3  objective J                       -> lks_forward (J_dev)
 *   Step 4  adjoint fields by ALKS            -> alks_adjoint
 *   Step 5  design sensitivity dJ/dgamma      -> lks_sensitivity
 * for the problem  min_gamma J(gamma, U(gamma)),  0 <= gamma <= 1  (Eq. obj).
 *
 * Conventions
 *  - Lattice units: dx = dt = 1.  D2Q9 lattice; nodes sit on the domain edges.
 *  - A field is an array of nx*ny values, node (i, j) at j*nx + i (x fastest),
 *    dense, in the element type `real_type` of the descriptor (float or double).
 *  - Pointers named *_dev are device pointers on the current device; *_host are
 *    host pointers (pageable or pinned).
 *  - Ownership: the caller owns every buffer it passes in, including the workspace
 *    given to lks_create.  The library allocates no device memory at any point and
 *    keeps no pointer to caller buffers beyond the call, except the workspace.
 *  - Every call is ordered on the CUDA stream given to lks_create and returns
 *    without synchronising, unless stated otherwise.
 *  - Errors: arguments are checked on the host before any launch; a failing check
 *    returns LKS_ERR_INVALID_ARG and launches nothing.  Conditions detected on the
 *    device (non-finite or runaway velocity) are recorded in a status word in the
 *    workspace and reported by the next call that synchronises (lks_query,
 *    lks_gradient_host).  Calls never throw.  lks_last_error gives a message.
 */
#ifndef LKS_H
#define LKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LKS_DESC_VERSION 3

typedef enum {
    LKS_OK = 0,
    LKS_ERR_INVALID_ARG = 1,   /* bad descriptor, size or pointer                 */
    LKS_ERR_WORKSPACE = 2,     /* workspace too small or misaligned               */
    LKS_ERR_CUDA = 3,          /* a CUDA runtime call failed                      */
    LKS_ERR_UNSTABLE = 4,      /* non-finite or |u| > 0.5 seen on the device       */
    LKS_ERR_NOT_CONVERGED = 5, /* a tolerance march (tol > 0) hit max_steps        */
    LKS_ERR_TIMEOUT = 6,       /* a bounded device wait gave up                    */
    LKS_ERR_STATE = 7          /* calls in the wrong order (e.g. adjoint first)    */
} lks_status;

typedef enum { LKS_REAL_F32 = 0, LKS_REAL_F64 = 1 } lks_real_type;

/* Storage type of checkpoint snapshots (unsteady problems). */
typedef enum { LKS_SNAP_F32 = 0, LKS_SNAP_BF16 = 1, LKS_SNAP_F16 = 2 } lks_snap_type;

/* How the marches run.  STEP: one kernel launch per time step (FP32 lattices with
 * nx % 4 == 0 stage their tiles by tensor copies; large non-thermal FP32 lattices,
 * with at least four column tiles per SM, use the warp-column kernels).  RESIDENT:
 * one cooperative launch per steady march in which every tile stays resident in
 * the shared memory of its CTA (lattices whose tiles fit the GPU at once).  COLUMN:
 * one launch per step of the warp-column kernels at any size (FP32, non-thermal,
 * nx % 4 == 0; otherwise as STEP).  AUTO: RESIDENT where it fits, else STEP.
 * D3Q19 lattices (FP32, nx % 4 == 0): STEP runs the forward and the adjoint on
 * the plane-march kernels; every other value runs both on the warp-column z-march
 * kernels. */
typedef enum {
  LKS_PATH_AUTO = 0,
  LKS_PATH_STEP = 1,
  LKS_PATH_RESIDENT = 2,
  LKS_PATH_COLUMN = 3
} lks_exec_path;

/* Thermal edge conditions (Sec. 2.4): prescribed temperature T = T_bar, or
 * prescribed heat flux -q.n = q_bar_w. */
typedef enum { LKS_T_FIXED = 0, LKS_T_FLUX = 1 } lks_thermal_kind;

/* Problem descriptor.  Geometry: inlet (prescribed velocity, parabola over the
 * span [in_y0, in_y1] of the left edge, zero elsewhere on that edge); pressure
 * outlet (rho = rho_out, tangential velocity zero) over [out_y0, out_y1] of the
 * right edge, walls elsewhere on the right edge; no-slip walls at the bottom and
 * top edges; corners are wall nodes. */
typedef struct {
    int32_t version;          /* LKS_DESC_VERSION                                   */
    int32_t nx, ny;           /* nodes per direction, >= 5                           */
    int32_t real_type;        /* lks_real_type of every field passed in or out       */
    double nu;                /* kinematic viscosity, Eq. (A): nu = (1/6 - 2A/9)     */
    double alpha_bar;         /* Brinkman interpolation, Eq. (brinkman)              */
    double q_alpha;
    double u_max;             /* inlet peak velocity                                */
    double pulse_mean;        /* u_in(t) = u_max (pulse_mean + pulse_amp sin(2 pi t / pulse_period)) */
    double pulse_amp;
    double pulse_period;      /* <= 0: steady inlet u_max * pulse_mean               */
    int32_t in_y0, in_y1;     /* inlet span, inclusive                               */
    int32_t out_y0, out_y1;   /* outlet span, inclusive, inside [1, ny-2];
                                 out_y1 = out_y0 - 1: no outlet (closed right wall) */
    double rho_out;           /* outlet density, p_bar = rho_out / 3                 */
    int32_t thermal;          /* 1: thermal lattice for T (Eqs. T, geq2)             */
    int32_t steady;           /* 1: steady (adjoint iterated on the final state)     */
    double K_f, K_s, q_K;     /* thermal diffusivity interpolation, Eq. (conductivity) */
    int32_t t_kind[4];        /* thermal condition per edge: left, right, bottom, top */
    double t_val[4];          /* T_bar or q_bar_w per edge                           */
    double kappa_T;           /* weight of the temperature term in the objective     */
    int32_t n_steps;          /* forward steps                                       */
    int32_t n_adj;            /* steady: adjoint iterations; unsteady: ignored       */
    int32_t checkpoint_every; /* unsteady: K > 0 recompute segments of K steps from
                                 snapshots (two segment stores in the workspace:
                                 the recompute of a segment overlaps the adjoint of
                                 the next); 0 keeps every level (plain form)         */
    int32_t snapshot_type;    /* lks_snap_type of the checkpoint snapshots           */
    int32_t exec_path;        /* lks_exec_path: 0 automatic, 1 one kernel launch per
                                 step, 2 resident persistent march (steady problems
                                 whose tiles fit on the GPU at once), 3 warp-column
                                 kernels per step                                    */
    int32_t lattice;          /* lks_lattice: 0 D2Q9 (default), 1 D3Q19 (see below)   */
    int32_t nz;               /* D3Q19: nodes along z, >= 5; D2Q9: 0 or 1            */
    int32_t res_steps;        /* resident marches: time steps per exchange of tile
                                 bands, 0 automatic or 1..3; the largest value up to
                                 this that fits the tile shape and shared memory runs */
    double kappa_p;           /* weight of the static pressure drop in J (Eq.
                                 objective_pipebend): J = J_O + kappa_p J_p with
                                 J_p = 1/3 (sum of rho over the inlet nodes - over
                                 the outlet nodes); the adjoint edge rule carries
                                 +kappa_p (inlet nodes) or -kappa_p (outlet nodes) in
                                 every residual row of Eqs. afboundaryu / afboundaryp.
                                 D2Q9: steady problems only; inlet nodes are the left
                                 edge nodes inside [in_y0, in_y1] (corners excluded),
                                 outlet nodes the pressure nodes.  D3Q19: see below */
    double tol;               /* steady D2Q9: > 0 marches to a relative step change
                                 of tol (see lks_forward); 0 fixed step counts        */
    int32_t max_steps;        /* tol > 0: step limit of each march (>= n_steps, n_adj) */
    int32_t warm_start;       /* steady D2Q9: 1 = lks_forward marches from the handle's
                                 current state (the last forward, lks_set_state or
                                 lks_march) instead of from rest, and alks_adjoint
                                 from the current adjoint fields instead of zero;
                                 with no earlier state it starts from rest.  The
                                 usual start inside an optimisation loop, where the
                                 design changes little between calls              */
    int32_t segment_type;     /* unsteady FP32: lks_snap_type of the stored levels
                                 of u, v[, T] that the adjoint reads -- the whole
                                 trajectory (checkpoint_every = 0) or the recomputed
                                 segment (checkpoint_every > 0).  F32 (default), or
                                 BF16 / F16 (half the bytes: each forward step's
                                 level is packed, each adjoint step's unpacked)     */
    int32_t reserved[4];      /* must be zero                                        */
    /* Thermal source terms (thermal = 1; they run on the per-step kernels, so
     * exec_path must be AUTO or STEP).  Heat source Q = beta_gamma (1 - T) of Eq.
     * (heatsource) with beta_gamma = beta_bar q_beta (1 - gamma) / (q_beta + gamma)
     * (Eq. betagamma), entering T once per step, implicitly:
     * T = (T* + beta_gamma) / (1 + beta_gamma) on interior nodes; its adjoint divides
     * T~ likewise and the sensitivity gains -beta' (1 - T) T~.  Heat-exchange
     * objective (Eq. objective_heatexchanger): J_O gains -kappa_Q beta_gamma (1 - T)
     * per interior node.  Boussinesq force G = g beta (T - T_ref) (Eq.
     * boussinesqforce; gb = the products g_x beta, g_y beta) with T of the new level:
     * u = (u* + G) / (1 + alpha_gamma); its adjoint adds 3 g beta . u~ to T~ (Eq.
     * albeg_ex).  All zero: none. */
    double beta_bar, q_beta;
    double kappa_Q;
    double gb[2];
    double T_ref;
    /* Heated segment of a heat-flux bottom edge (t_kind[2] = LKS_T_FLUX): the nodes
     * heat_x0 <= i <= heat_x1 of the bottom edge carry the flux heat_q instead of
     * t_val[2] (the paper's heat sink: a short heated part of an otherwise adiabatic
     * wall).  heat_x1 < heat_x0: none. */
    int32_t heat_x0, heat_x1;
    double heat_q;
    /* Energy loss (Eq. objective_doublepipe), D2Q9: J gains kappa_E J_E with J_E the
     * outflow of total pressure, the sum over the inlet nodes (as for kappa_p) and the
     * outlet nodes of -n.u (p + |u|^2 / 2), p the pressure above the outlet's,
     * (rho - rho_out) / 3; unsteady problems sum it over levels 1..n_steps.  The
     * adjoint edge rule carries kappa_E u in every residual row of the inlet nodes
     * (the integrand's derivative with respect to p) and, on the outlet nodes,
     * 3 kappa_E (-3/2 u_n^2) (c_i.n) / rho_out (three times its derivative with
     * respect to f_i through u_n).  Runs on the per-step kernels (exec_path AUTO or
     * STEP).  0: none. */
    double kappa_E;
} lks_problem_desc;

/* Three dimensions (lattice = LKS_LATTICE_D3Q19).  The paper states LKS / ALKS in
 * two dimensions (Secs. 2.4-2.5) and names three as the extension (Sec. 4); the
 * D3Q19 form writes the same equations for 19 velocities (w = 1/3, 1/18, 1/36;
 * nu = 1/6 - 2A/9 unchanged).  Geometry: a duct, inlet over the face x = 0 with
 * u_x = u_max 16 y(1-y) z(1-z) (y, z scaled to [0, 1]), prescribed pressure on the
 * face x = nx-1, walls on the four side faces; nodes on two or three faces are wall
 * nodes.  Steady and non-thermal only (steady = 1, thermal = 0); the inlet and
 * outlet spans, pulse, thermal and checkpoint fields are ignored.  Objective:
 * J = J_O + kappa_p J_p with the total dissipation J_O and the static pressure drop
 * J_p = 1/3 (sum of rho over the inlet nodes - over the outlet nodes) of Eq.
 * objective_pipebend (p = rho / 3, dGamma = 1, nodes on one face only); the adjoint
 * edge rule carries +kappa_p (inlet) or -kappa_p (outlet) in every residual row of
 * Eqs. afboundaryu / afboundaryp.  Fields are
 * nx*ny*nz values, x fastest, then y, then z.  lks_get_state returns w through its
 * T pointer; alks_get_adjoint fills 10 fields (rho~, u~x, u~y, u~z, s~xx, s~xy,
 * s~xz, s~yy, s~yz, s~zz).  lks_set_state, lks_march, alks_set_adjoint, alks_march
 * and lks_gradient_noalloc answer LKS_ERR_INVALID_ARG for a D3Q19 handle. */
typedef enum { LKS_LATTICE_D2Q9 = 0, LKS_LATTICE_D3Q19 = 1 } lks_lattice;

/* Counters and the device status word, filled by lks_query. */
typedef struct {
    int64_t forward_steps;    /* forward steps launched since create (incl. recompute) */
    int64_t adjoint_steps;    /* adjoint steps launched since create                 */
    int64_t kernel_launches;  /* kernels launched since create                       */
    size_t workspace_bytes;   /* workspace in use                                    */
    int32_t device_status;    /* lks_status recorded on the device (0 = none)        */
    int32_t phase;            /* 0 created, 1 forward done, 2 adjoint done           */
    int32_t fwd_path;         /* lks_exec_path the last forward march ran on         */
    int32_t adj_path;         /* lks_exec_path the last adjoint march ran on         */
    int32_t res_steps_fwd;    /* steps per band exchange of the last resident forward
                                 march (0: none ran)                                  */
    int32_t res_steps_adj;    /* the same for the last resident adjoint march        */
    double fwd_change;        /* tol > 0: relative change of the last measured forward
                                 step (0: none measured)                              */
    double adj_change;        /* the same for the adjoint                            */
} lks_stats;

typedef struct lks_handle lks_handle;

/* Workspace bytes for a problem (host only, pure).  Errors: LKS_ERR_INVALID_ARG
 * for a bad descriptor. */
lks_status lks_workspace_size(const lks_problem_desc *desc, size_t *bytes);

/* Creates a handle on the current device.  workspace_dev: caller-owned device
 * memory of at least lks_workspace_size bytes, 256-byte aligned, kept alive and
 * unused by the caller until lks_destroy.  stream: a cudaStream_t (NULL = legacy
 * default stream).  Host allocation of the handle itself only; for unsteady
 * problems with checkpoint_every > 0 the handle also creates one non-blocking
 * stream and five events of its own (destroyed by lks_destroy), on which
 * alks_adjoint runs the segment recomputations (see alks_adjoint).  Returns
 * LKS_ERR_CUDA if they cannot be created. */
lks_status lks_create(const lks_problem_desc *desc, void *workspace_dev, size_t bytes,
                      void *stream, lks_handle **out);

/* Step 2 + 3 (Sec. 2.4, Eqs. rho, u, T with feq2, geq2, lbef_ex; objective Eq. fj):
 * marches the state from rest (rho = 1, u = 0, T = 0) for n_steps steps with the
 * design field gamma_dev (nx*ny, real_type, values in [0, 1]; copied into the
 * workspace) and writes the objective J to J_dev (one double, device).  Steady: J
 * is J_O of the final state.  Unsteady: J is the sum of J_O over levels 1..n_steps;
 * snapshots or the full trajectory are kept for the adjoint.  J_O is the total
 * dissipation over interior nodes, sum nu/2 S:S + alpha_gamma |u|^2, plus kappa_T T.
 * Steady D2Q9 with tol > 0: after the n_steps steps one more step is taken and its
 * relative change r = max(|du| + |dv|) / max(|u| + |v|) measured (the flow only;
 * a thermal T is not part of the measure); chunks of n_steps
 * steps and a measured step repeat until r <= tol or max_steps steps have run.  If
 * the limit comes first the call returns LKS_ERR_NOT_CONVERGED with the state and J
 * of the last step in place (lks_query reports r as fwd_change). */
lks_status lks_forward(lks_handle *h, const void *gamma_dev, double *J_dev);

/* Step 4 (Sec. 2.5, Eqs. ap-aq, afeq, ageq, albef_ex, ftilde; App. A): the ALKS
 * march from the terminal condition (Eqs. afinitial, aginitial) with the
 * generalized-inverse edge rule.  Steady: n_adj iterations on the final state.
 * Unsteady: backward over all levels (recomputing segments from snapshots when
 * checkpoint_every > 0) and the sensitivity accumulated on the way.  With
 * checkpoints, segment s - 1 is recomputed on the handle's own stream while the
 * adjoint marches segment s on the caller's stream (events order the two; the
 * results are those of recomputing and marching one segment after the other); the
 * call returns with the caller's stream waiting for all of that work.
 * Steady D2Q9 with tol > 0: iterations in chunks of n_adj, each followed by one
 * measured iteration (the relative change of u~, as for lks_forward), until the
 * change is <= tol or max_steps iterations have run (LKS_ERR_NOT_CONVERGED, the
 * adjoint of the last iteration in place; adj_change in lks_query).
 * LKS_ERR_STATE if lks_forward has not run. */
lks_status alks_adjoint(lks_handle *h);

/* Step 5 (Sec. 2.5, the integrand of <J', dgamma>): writes dJ/dgamma (nx*ny,
 * real_type, device) = dJ_O/dgamma + 3 alpha' u.u~ - B' grad T . q~ on interior
 * nodes (summed over levels when unsteady) and 0 on edge nodes.  LKS_ERR_STATE if
 * alks_adjoint has not run. */
lks_status lks_sensitivity(lks_handle *h, void *dJdgamma_dev);

/* Steps 2-5 end to end with host buffers: copies gamma_host to the device, runs
 * lks_forward, alks_adjoint and lks_sensitivity, copies J and dJ/dgamma back and
 * synchronises the stream.  Returns the device status word if it is set. */
lks_status lks_gradient_host(lks_handle *h, const void *gamma_host, double *J_host,
                             void *dJdgamma_host);

/* State access for tests and tools: fields (nx*ny, real_type, device) drho, u, v, T
 * where drho = rho - 1 is the density deviation the library stores (T ignored
 * unless thermal).  lks_set_state also sets the time level t of the state (the
 * inlet pulse of the next step uses t + 1); gamma_dev as in lks_forward. */
lks_status lks_set_state(lks_handle *h, const void *gamma_dev, const void *drho_dev,
                         const void *u_dev, const void *v_dev, const void *T_dev, int32_t t);
lks_status lks_get_state(lks_handle *h, void *drho_dev, void *u_dev, void *v_dev, void *T_dev);

/* n forward steps from the current state (no objective, no snapshots). */
lks_status lks_march(lks_handle *h, int32_t n);

/* Adjoint fields (9 arrays of nx*ny, real_type, device, in the order rho~, u~_x,
 * u~_y, s~_xx, s~_xy, s~_yy, T~, q~_x, q~_y; the thermal three are ignored unless
 * thermal). */
lks_status alks_set_adjoint(lks_handle *h, void *const *fields_dev);
lks_status alks_get_adjoint(lks_handle *h, void *const *fields_dev);

/* n ALKS steps from the current adjoint fields with the state frozen at the
 * current state (the steady iteration of alks_adjoint). */
lks_status alks_march(lks_handle *h, int32_t n);

/* Counters and device status (synchronises the stream). */
lks_status lks_query(lks_handle *h, lks_stats *out);

/* Destroys the handle (host memory only; the workspace stays the caller's). */
lks_status lks_destroy(lks_handle *h);

/* Static message for a status; last error message of a handle (never NULL). */
const char *lks_status_string(lks_status s);
const char *lks_last_error(const lks_handle *h);

/* Steps 2-5 without any device allocation, for callers that cannot call cudaMalloc
 * and cannot hand the library a workspace: a plugin whose host application owns all
 * device memory through a fixed pool, or a latency-critical loop in which the
 * implicit synchronisation of cudaMalloc / cudaFree is not allowed.  The paper has
 * no counterpart; this is a packaging variant of lks_forward + alks_adjoint +
 * lks_sensitivity (same kernels, same results).
 *
 * The workspace comes from one static device array of LKS_NOALLOC_SCRATCH_BYTES
 * (8 MiB) inside the library; every GPU that loads the library holds it until the
 * process exits.  A problem whose lks_workspace_size exceeds it is rejected with
 * LKS_ERR_WORKSPACE before any GPU work (about 100 000 nodes fit for a steady FP32
 * problem, e.g. 256 x 256).  gamma_dev, J_dev (one double) and dJdgamma_dev
 * (nx*ny, real_type) are the caller's device buffers; stream orders the work.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  Every call shares the array and leaves its contents behind (each
 * call clears what it needs zeroed), so calls that overlap on the GPU -- on
 * different streams, or from different host threads -- race and corrupt each
 * other: order them.  Host memory for a temporary handle is still allocated.
 * Descriptors with tol > 0 are rejected (LKS_ERR_INVALID_ARG): a tolerance march
 * reads its measured change back to the host.
 * Errors: the return value covers what the host can see (arguments, size, launch
 * failures); this entry point keeps no handle, so lks_last_error has no message for
 * it.  A condition the kernels detect on the device (non-finite or runaway velocity,
 * a bounded wait that gave up) cannot be returned without synchronising; the call
 * then overwrites *J_dev with a quiet NaN after the gradient, so a caller that
 * checks J for NaN sees every device-detected failure (dJdgamma is not valid then).
 * Nothing the call enqueues reads host memory after it returns. */
#define LKS_NOALLOC_SCRATCH_BYTES ((size_t)8 << 20)
lks_status lks_gradient_noalloc(const lks_problem_desc *desc, const void *gamma_dev, double *J_dev,
                                void *dJdgamma_dev, void *stream);

/* Host-only: the edge-class moment maps used by the adjoint kernels, for checks on
 * a CPU.  cls: 0 left face, 1 right pressure face, 2 right wall face, 3 bottom
 * face, 4 top face, 5..8 corners (bottom-left, bottom-right, top-left, top-right).
 * out: 6 x 10 doubles, row r = moment r (rho~, u~_x, u~_y, s~_xx, s~_xy, s~_yy) as a
 * linear function of the nine gathered f~ (columns 0..8; unknown entries ignored)
 * and of the heat-flux coupling kappa~ T (column 9).  Eq. (ftilde) generalised to
 * every face by the least squares of Sec. 2.5 (Eqs. afboundaryu, afboundaryp,
 * afboundaryuq, afboundarypq). */
lks_status lks_edge_moment_map(double A, int32_t cls, double *out);

/* Host-only: the response of the six flow moments of an edge node of class cls to a
 * unit boundary objective term added to every residual row (dJ_dO/df_i of Eqs.
 * afboundaryu / afboundaryp, with the known f~ and kappa~ T zero).  The adjoint
 * kernels add kappa_p times this (+ on inlet nodes, - on outlet nodes) for the
 * static pressure drop.  out: 6 doubles. */
lks_status lks_edge_objective_map(double A, int32_t cls, double *out);

/* Diagnostics: runs one of the library's bounded device waits on a condition that
 * never comes true, on cuda_stream, and returns in *recorded the status the kernel
 * wrote: LKS_ERR_TIMEOUT when the wait gave up as designed.  which: 0 the tile-flag
 * wait of the resident marches (about 2 s), 1 the mbarrier wait of the TMA-staged
 * kernels (well under a second).  scratch_dev: 2 int32 of device memory owned by the
 * caller, overwritten.  Synchronises the stream.  A wait that gives up returns (it
 * does not trap), so the CUDA context stays usable.  Errors: LKS_ERR_INVALID_ARG for
 * a bad which or a NULL pointer (before any GPU work), LKS_ERR_CUDA. */
lks_status lks_selftest_wait(int32_t which, int32_t *scratch_dev, void *cuda_stream, int32_t *recorded);

/* ---------------------------------------------------------------------------------
 * Batched form: many designs (load cases, optimiser candidates) of unequal lattice
 * size marched in lock step.  One persistent launch per time step covers every
 * tile of every design, and the whole gradient (Steps 2-5 of Sec. 2.7 for all
 * designs: forward march with checkpoints, objective, checkpointed adjoint with
 * segment recomputation, sensitivity) is one CUDA graph launch.  The paper runs one
 * design at a time; this is the same per-node computation as lks_forward +
 * alks_adjoint + lks_sensitivity of an unsteady FP32 problem with
 * checkpoint_every = K, applied to each design.
 *
 * Scope: unsteady, non-thermal, FP32 designs that share n_steps.  Each descriptor
 * passes the lks_create checks; its checkpoint_every, snapshot_type and exec_path
 * are ignored (the batch options rule).  nx need not be a multiple of 4.
 *
 * Layout: the designs' lattices are packed side by side into one arena per field
 * (shelf packing of rectangles whose extents are rounded up to 128 x 16 nodes), so
 * a single tensor map per field serves every design; a work list names each
 * (design, tile) pair.  The tile shape of the TMA-staged kernels is one of
 * LKS_BATCH_TILE_CONFIGS fixed shapes, picked by timing each on the batch at
 * lks_batch_create (tile_config = -1) or given; the forward and the adjoint may
 * instead run the warp-column kernels (fwd_column, adj_column), again timed or given.  K = 0 picks the checkpoint spacing that minimises workspace bytes
 * (snapshots + segment buffer), a pure function of the descriptors.
 * --------------------------------------------------------------------------------- */
#define LKS_BATCH_VERSION 1
#define LKS_BATCH_TILE_CONFIGS 4
typedef struct lks_batch lks_batch;

typedef struct {
  int32_t version;          /* LKS_BATCH_VERSION */
  int32_t checkpoint_every; /* K >= 1, or 0: memory-optimal K */
  int32_t snapshot_type;    /* lks_snap_type of the checkpoints (per design and field max-abs scale) */
  int32_t tile_config;      /* -1: autotune at create; else 0 .. LKS_BATCH_TILE_CONFIGS - 1:
                               0 = 64x8, 1 = 32x16, 2 = 128x4, 3 = 64x16 output nodes per tile */
  int32_t use_graph;        /* 1: each gradient is one CUDA graph launch; 0: direct launches */
  int32_t fwd_column;       /* forward kernel: -1 the faster of the two, timed at create; 0 the
                               TMA-staged kernel at tile_config; 1 the warp-column kernel
                               (60 x 40 tiles, two columns per lane)                  */
  int32_t adj_column;       /* adjoint kernel: -1 the faster of the two, timed at create; 0 the
                               TMA-staged kernel at tile_config; 1 the warp-column kernel
                               (28 x 32 tiles)                                        */
  int32_t reserved[5];      /* must be zero */
} lks_batch_options;

typedef struct {
  int32_t n_designs;
  int32_t tile_config;      /* the shape in use */
  int32_t checkpoint_every; /* K in use */
  int32_t n_ckpt;
  int32_t arena_w, arena_h; /* arena extent in nodes */
  int32_t graph;            /* 1 when a gradient is one graph launch */
  int32_t device_status;    /* lks_status the kernels recorded (0 = none) */
  int64_t nodes;            /* sum of nx * ny over the designs */
  int64_t ntiles;           /* work-list length at the tile shape in use */
  int64_t workspace_bytes;
  int64_t kernel_launches;  /* kernels one gradient launches (inside the graph when used) */
  int64_t gradients;        /* gradients computed so far */
  float tune_us[LKS_BATCH_TILE_CONFIGS]; /* autotuner: us per level of each shape, two forward steps
                                            (march, recompute) + one adjoint step (0: not timed) */
  int32_t fwd_column;       /* 1 when the forward runs the warp-column kernel */
  float tune_fwd_us[LKS_BATCH_TILE_CONFIGS]; /* autotuner: us per forward step of each shape (0: not timed) */
  float tune_col_us;        /* autotuner: us per forward step of the warp-column kernel (0: not timed) */
  int32_t adj_column;       /* 1 when the adjoint runs the warp-column kernel */
  float tune_acol_us;       /* autotuner: us per adjoint step of the warp-column kernel (0: not timed);
                               the (shape, forward kernel, adjoint kernel) of least per-level time
                               is used */
} lks_batch_stats;

/* Host only.  n designs described by descs[0..n-1]; opt as above (NULL: K = 0,
 * BF16 snapshots, autotuned tile, graph).  *bytes: device workspace to pass to
 * lks_batch_create. */
lks_status lks_batch_workspace_size(int32_t n, const lks_problem_desc *descs, const lks_batch_options *opt,
                                    size_t *bytes);
/* Lays out the arena and the work lists, uploads per-design tables, autotunes the
 * tile shape when asked (running short marches on a uniform design) and captures
 * the gradient graph, in which the recompute of a checkpoint segment is a branch
 * parallel to the adjoint of the next segment (captured on a non-blocking stream
 * the batch handle creates, with five events; destroyed by lks_batch_destroy).
 * workspace: caller-owned device memory of at least the size above, 256-byte
 * aligned (two segment stores); never freed by the library.  Synchronises the
 * stream.  Returns LKS_ERR_CUDA if the stream or events cannot be created. */
lks_status lks_batch_create(int32_t n, const lks_problem_desc *descs, const lks_batch_options *opt,
                            void *workspace, size_t bytes, void *cuda_stream, lks_batch **out);
/* All designs' gradients.  gamma_dev: host array of n device pointers to each
 * design's gamma (ny x nx FP32, row-major, read only).  J_dev: device array of n
 * doubles (objective of each design).  dJdgamma_dev: host array of n device
 * pointers (ny x nx FP32, written).  Stream-ordered: returns after enqueueing; the
 * host arrays may be reused at once.  Device-detected errors (instability, a
 * timed-out wait) are reported by lks_batch_query. */
lks_status lks_batch_gradient(lks_batch *b, const float *const *gamma_dev, double *J_dev,
                              float *const *dJdgamma_dev);
/* Synchronises the stream and fills *out. */
lks_status lks_batch_query(lks_batch *b, lks_batch_stats *out);
lks_status lks_batch_destroy(lks_batch *b);
const char *lks_batch_last_error(const lks_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* LKS_H */
