/*
 * idugks.h -- C ABI of libidugks, a GB300 (sm_103a) implementation of one
 * iteration of the implicit discrete unified gas-kinetic scheme (IDUGKS) of
 * Pan, Zhong & Zhuo, "An Implicit Discrete Unified Gas-Kinetic Scheme for
 * Simulations of Steady Flow in All Flow Regimes", arXiv 1709.01819.
 *
 * The problem statement follows Section 2 of the paper: a 2-D BGK or
 * BGK-Shakhov gas (Eq. 1-7, 20) on a structured quadrilateral block, discrete
 * velocities from a Gauss-Hermite or Newton-Cotes rule (Section 2.2, last
 * paragraph), diffuse walls and far-field ghosts (Section 2.3, Eq. 34-35).
 * One call to idg_iterate performs, per iteration: the DUGKS interface flux
 * (Eq. 10-19), the macroscopic LU-SGS predictor (Eq. 27-31) and the
 * matrix-free LU-SGS sweeps for the distribution (Eq. 22-26), then the update
 * of Eq. (32).
 *
 * Conventions
 *  - Units: reference density 1, reference length 1, velocity unit
 *    sqrt(2 R T_ref).  Temperatures are in units of T_ref; RT_ref is set by
 *    idg_set_gas (1/2 in this unit system).
 *  - Every function returns an idg_status.  On failure idg_last_error(ctx)
 *    gives a one-line reason.  No function traps or aborts; device-side
 *    problems surface as IDG_ERR_NONFINITE or IDG_ERR_CUDA.
 *  - Host arrays are owned by the caller and copied during the call.
 *  - Device memory comes from one caller-owned workspace (idg_workspace_size,
 *    idg_bind_workspace); the library allocates no device memory itself.
 *    The workspace must stay valid until idg_destroy or the next bind.
 *  - All device work is ordered on the caller's CUDA stream (cudaStream_t
 *    passed as void*; NULL is the legacy default stream).  Functions that
 *    return host data synchronise that stream.
 *  - Setters are accepted until idg_bind_workspace; afterwards they return
 *    IDG_ERR_STATE.
 *  - Layouts: cell index c = j*ni + i; mesh node index j*(ni+1) + i; discrete
 *    velocity index k = ky*nvx + kx; per-(cell, velocity) host arrays are
 *    [cell][velocity] row-major float64.
 */
#ifndef IDUGKS_H
#define IDUGKS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct idg_ctx idg_ctx;

typedef enum {
    IDG_OK = 0,
    IDG_ERR_ARG = 1,           /* invalid argument (size, range, NULL)                 */
    IDG_ERR_STATE = 2,         /* call not allowed in the context's current state      */
    IDG_ERR_CUDA = 3,          /* a CUDA runtime call failed                           */
    IDG_ERR_OOM = 4,           /* workspace smaller than idg_workspace_size            */
    IDG_ERR_NONFINITE = 5,     /* the residual became NaN or Inf (sticky until the     */
                               /* next idg_init_uniform or idg_set_state)              */
    IDG_ERR_TIMEOUT = 6,       /* reserved: no kernel of this library waits on another */
                               /* thread block, so none is returned                    */
    IDG_ERR_NOT_CONVERGED = 7  /* idg_iterate reached max_iter above tol               */
} idg_status;

enum { IDG_FP64 = 0, IDG_MIXED = 1 };              /* storage/compute precision of f   */
enum { IDG_BC_PERIODIC = 0, IDG_BC_WALL = 1, IDG_BC_FARFIELD = 2 };
enum { IDG_NC_TRAP = 0, IDG_NC_SIMPSON = 1, IDG_GAUSS_HERMITE = 2 };
enum { IDG_IMIN = 0, IDG_IMAX = 1, IDG_JMIN = 2, IDG_JMAX = 3 };
enum { IDG_BGK = 0, IDG_SHAKHOV = 1 };

/* Create a context.  precision: IDG_FP64 (f stored and processed in float64)
 * or IDG_MIXED (f in float32; moments, macroscopic predictor and residual in
 * float64).  device: CUDA ordinal used by later calls.  No GPU work happens
 * here.  *out receives a context owned by the caller (free with idg_destroy). */
idg_status idg_create(idg_ctx **out, int precision, int device);
void idg_destroy(idg_ctx *ctx);
const char *idg_last_error(const idg_ctx *ctx);

/* Structured quadrilateral block of ni x nj cells (Fig. 1 and Section 2.3),
 * min(ni, nj) <= 256 (a larger block is refused with IDG_ERR_ARG by
 * idg_workspace_size and idg_bind_workspace).
 * nodes_x/nodes_y: (ni+1)*(nj+1) host float64, node (i,j) at j*(ni+1)+i, cells
 * counter-clockwise (positive area).  A periodic direction is declared with
 * idg_set_boundary(kind = IDG_BC_PERIODIC) on both of its sides; the last node
 * column/row then equals the first up to a constant translation. */
idg_status idg_set_mesh_structured(idg_ctx *ctx, int ni, int nj, const double *nodes_x,
                                   const double *nodes_y);

/* Unstructured mesh of triangles and quadrilaterals (the hybrid meshes of
 * Section 3), in place of a structured block.
 *  - x, y: nnodes host float64 node coordinates.
 *  - cell_nodes: host [ncells][4] node indices, counter-clockwise (positive
 *    area); -1 as the 4th entry of a triangle.  Slot m of a cell is its edge
 *    from node m to node m+1; two cells sharing an edge must run along it in
 *    opposite directions.
 *  - edge_side: host [ncells][4]: for a slot whose edge has no neighbour, the
 *    boundary group 0..3 whose idg_set_boundary condition applies (a wall or
 *    the far field; periodic is refused: close a ring by sharing its nodes);
 *    ignored elsewhere (-1 allowed).
 * The cell numbering is the LU-SGS order (Eq. 26, 30: lower neighbours are
 * those of smaller index); the sweeps run level by level through it.  A cell
 * without two neighbours in independent directions gets no least-squares
 * gradient (first-order reconstruction).  Faces are numbered in order of first
 * appearance (cell by cell, slot by slot).  Malformed meshes are refused at
 * idg_bind_workspace (IDG_ERR_ARG).  Such a context cannot run idg_adjoint or
 * join a batch (IDG_ERR_ARG).  At most 2^24 cells. */
idg_status idg_set_mesh_unstructured(idg_ctx *ctx, int nnodes, const double *x, const double *y, int ncells,
                                     const int *cell_nodes, const int *edge_side);

/* Tensor-product discrete velocity grid (Section 2.2, closing paragraph).
 * IDG_NC_TRAP: composite trapezoid (closed 2-point Newton-Cotes) on
 * [xmin,xmax] x [ymin,ymax], any n >= 2.  IDG_NC_SIMPSON: composite Simpson,
 * odd n >= 3.  IDG_GAUSS_HERMITE: nodes scaled by sqrt(2 RT_ref), ranges
 * ignored.  At most 16384 velocities in total. */
idg_status idg_set_velocity_grid(idg_ctx *ctx, int rule, int nx, int ny, double xmin,
                                 double xmax, double ymin, double ymax);

/* Gas (Eq. 1-7, 20, 36): K internal degrees of freedom, Prandtl number (used
 * by IDG_SHAKHOV), viscosity exponent omega (mu ~ T^omega), Knudsen number
 * defining mu_ref by the VHS mean free path, RT_ref, model IDG_BGK/IDG_SHAKHOV. */
idg_status idg_set_gas(idg_ctx *ctx, int K, double Pr, double omega, double Kn, double RT_ref,
                       int model);

/* Boundary of one side (Section 2.3).  IDG_BC_WALL: diffuse wall with velocity
 * (u, v) and temperature T (Eq. 34-35); rho ignored.  IDG_BC_FARFIELD: incoming
 * particles from the Maxwellian (rho, u, v, T).  IDG_BC_PERIODIC: set on both
 * sides of a direction. */
idg_status idg_set_boundary(idg_ctx *ctx, int side, int kind, double rho, double u, double v,
                            double T);

/* Numerics: cfl_imp sets the per-cell pseudo time step dt_imp = cfl_imp h_i /
 * xi_max of Eq. (26) and (30); cfl_phys the physical DUGKS step dt = cfl_phys
 * h_min / xi_max of Eq. (8); limiter 0 (phi = 1) or 1 (Eq. 16-17);
 * lusgs_omega the relaxation of the macroscopic LU-SGS (2 reproduces Eq. 30);
 * flags 0 or IDG_NUM_EXPLICIT.
 * IDG_NUM_EXPLICIT: idg_iterate and idg_iterate_profiled advance explicit
 * DUGKS time steps instead of IDUGKS iterations: the cell and face stages of
 * the iteration (Eq. 10-20, flux with the physical step dt) followed by the
 * update of Eq. (21), f~ <- (2tau-dt)/(2tau+dt) f~ + 2dt/(2tau+dt) f^S -
 * dt/Omega sum_faces F, tau and f^S at the moments of f~.  W is the moment
 * set of f~ (recomputed before the first step of every call and after each
 * step); cfl_imp and lusgs_omega are unused.  The residual of a step is
 * ||(W^{n+1} - W^n)/dt||_2 (at the fixed point of the march R_W balances the
 * moments of the discrete collision term and does not vanish).  Such a
 * context can neither join a batch nor run idg_adjoint (IDG_ERR_ARG). */
enum { IDG_NUM_EXPLICIT = 1 };
idg_status idg_set_numerics(idg_ctx *ctx, double cfl_imp, double cfl_phys, int limiter,
                            double lusgs_omega, int flags);

/* Smoothing constant K of the Venkatakrishnan limiter (Eq. 16-17, limiter
 * 1 of idg_set_numerics).  K = 0 (default): the limiter as the paper prints
 * it, whose factor drops to 0 wherever a cell value is its neighbourhood's
 * extremum.  K > 0: the form of the limiter's source (Venkatakrishnan's
 * steady-convergence paper, which the paper cites), each face's factor
 *     (P^2 + eps^2 + 2 D P) / (P^2 + 2 D^2 + P D + eps^2),
 * D the unlimited extrapolated increment to the face, P the increment to the
 * neighbourhood's max (D > 0) or min (D < 0), eps^2 = (K h)^3 with h the
 * square root of the cell's area; eps = 0 is Eq. 17's theta(P / D).  It
 * removes the limiter's switching at extrema, which can hold a steady
 * iteration in a limit cycle (and makes the limiter's derivative bounded for
 * idg_adjoint); too large a K under-limits shocks.  K >= 0, finite; before
 * idg_bind_workspace. */
idg_status idg_set_limiter_smoothing(idg_ctx *ctx, double K);

/* Macroscopic predictor of the implicit iteration (Eq. 28-31).  relax_sweeps
 * 0 (default): the LU-SGS forward and backward sweeps of Eq. (30).
 * relax_sweeps n in 1..64: point relaxation of the same predictor equations,
 * the other predictor the paper's conclusions name:
 *     D dW_c + sum_nb 1/2 (dF_nb S - omega Lambda dW_nb) = R_c,
 * solved by n Jacobi sweeps from dW = 0 (n = 1: dW = R / D), every cell in
 * parallel from the previous sweep.  Either predictor leaves the fixed point
 * (R_W = 0) unchanged; they differ in convergence per iteration and in cost
 * (LU-SGS is a dependent wavefront of 2(ni+nj-1) steps on one SM, each
 * relaxation sweep one grid-wide kernel).  A context with n > 0 cannot run
 * idg_adjoint, and the instances of a batch must share n (IDG_ERR_ARG).
 * Before idg_bind_workspace. */
idg_status idg_set_predictor(idg_ctx *ctx, int relax_sweeps);

/* Linearised diffuse wall in the micro sweeps (Section 2.3, Eq. 33-35).
 * on = 0 (default): ghost increments are zero in both sweeps, the start the
 * paper prescribes.  on = 1: the ghost cell of each wall face takes, in the
 * velocities coming into the domain, the increment drho_g M_w (Eq. 34; M_w
 * the wall's unit-density Maxwellian with the wall's velocity and
 * temperature, H part K RT_w G), with drho_g (Eq. 35) returning through the
 * wall the mass flux of the inner cell's outgoing increments of the previous
 * iteration (zero for the first iteration after idg_init_uniform or
 * idg_set_state).  The known ghost increment enters both sweeps as the
 * upwind neighbour term |xi.n| S Delta_ghost on the wall cells' right-hand
 * side; the face flux moments and R_W (the residual) exclude it, and the
 * fixed point is unchanged.  Far-field ghosts and the macroscopic predictor
 * keep zero ghost increments.  Call before idg_bind_workspace (else
 * IDG_ERR_STATE); on outside {0, 1}: IDG_ERR_ARG.  Such a context can join no
 * batch and run no idg_adjoint, and binding it with IDG_NUM_EXPLICIT set
 * fails (IDG_ERR_ARG). */
idg_status idg_set_implicit_wall(idg_ctx *ctx, int on);

/* Bytes of device workspace the configured problem needs (>= 0; host only). */
idg_status idg_workspace_size(idg_ctx *ctx, size_t *bytes);

/* Bind a caller-owned device buffer of at least idg_workspace_size bytes,
 * 256-byte aligned, on the context's device.  Uploads geometry and velocity
 * tables (synchronous).  Ends the setter phase. */
idg_status idg_bind_workspace(idg_ctx *ctx, void *dev_ptr, size_t bytes);

/* Uniform Maxwellian start (Section 3): W = exact moments of (rho, u, v, T),
 * f~ = discrete equilibrium.  Also fixes the reference Maxwellian the storage
 * is taken relative to.  Resets the iteration count and residual history. */
idg_status idg_init_uniform(idg_ctx *ctx, double rho, double u, double v, double T,
                            void *stream);

/* Replace / read the state.  G, H: host [ncell][nvel] float64 of f~ (Eq. 10),
 * W: host [ncell][4] float64 conservative variables (Eq. 4).  Any pointer may
 * be NULL in idg_get_state.  idg_set_state reads page-locked host arrays that
 * the CUDA runtime maps into the device's address space (cudaHostAlloc,
 * cudaHostRegister) in place, from its conversion kernel; other host memory
 * is first copied to a device staging buffer.  The result is the same. */
idg_status idg_set_state(idg_ctx *ctx, const double *G, const double *H, const double *W,
                         void *stream);
idg_status idg_get_state(idg_ctx *ctx, double *G, double *H, double *W, void *stream);

/* Checkpoint to / restart from a file (host I/O, synchronous on stream).
 * idg_save writes a 48-byte header -- the 8 bytes "IDGCKPT1", int32 format
 * version 2, int32 precision, int64 ncell, int64 nvel, int64 iterations
 * since the last restart, int64 hash of the discretisation (64-bit FNV-1a
 * of the mesh nodes and cell lists, the discrete velocities and weights and
 * K, top bit cleared) -- then, all float64 little-endian: G, H [ncell][nvel]
 * and W [ncell][4] (the idg_get_state view); the reference Maxwellian (rho,
 * u, v, T) the storage is taken relative to; and the stored deviations
 * f~ - M_ref of G and H [ncell][nvel].  idg_load checks the header against
 * the context (same cell and velocity counts and, for version 2, the same
 * discretisation hash; gas, boundaries and numerics may differ, e.g. to
 * continue a converged state at another Kn), restores that reference
 * Maxwellian and the deviations and W as stored, and restarts the residual
 * history as idg_set_state does: a context of the saving precision resumes
 * bitwise, one of the other precision converts the deviations to its
 * storage (the header's precision says which saved it).  Both need a bound
 * context (IDG_ERR_STATE); a null path, an unopenable, short, foreign or
 * mismatched file gives IDG_ERR_ARG. */
idg_status idg_save(idg_ctx *ctx, const char *path, void *stream);
idg_status idg_load(idg_ctx *ctx, const char *path, void *stream);

/* Run IDUGKS iterations (Section 2.2) until the residual ||R_W/Omega||_2
 * (explicit DUGKS: ||(W^{n+1} - W^n)/dt||_2, see IDG_NUM_EXPLICIT)
 * divided by that of the first iteration after the last (re)start is <= tol,
 * or max_iter iterations ran.  tol <= 0 runs exactly max_iter iterations.
 * iters_done and residual (relative) may be NULL.  Returns
 * IDG_ERR_NOT_CONVERGED when tol > 0 was not reached. */
idg_status idg_iterate(idg_ctx *ctx, int max_iter, double tol, void *stream, int *iters_done,
                       double *residual);

/* Per cell: rho, u, v, T/T_ref from W and the heat flux qx, qy of f from f~
 * (host [ncell][6] float64). */
idg_status idg_get_moments(idg_ctx *ctx, double *out6, void *stream);

/* Same output as idg_get_moments, written to device memory, for callers that
 * must not allocate device memory for it: real-time loops whose device memory
 * is fixed up front (an allocation there can stall or fail mid-run), or
 * plug-ins living inside another framework's memory pool (which owns every
 * allocation on the device and does not expect a library to make its own).  The call allocates nothing: its per-cell scratch (raw moments) is a
 * static device array of the library, 1.375 MiB on every GPU that loads
 * libidugks, kept until the process exits.  The paper has no counterpart; this
 * is a service of the library.
 *  - out6_dev: device memory of the context's device, [ncell][6] float64
 *    (rho, u, v, T/T_ref, qx, qy); the call is asynchronous on `stream`.
 *  - Meshes of more than 16384 cells are rejected with IDG_ERR_ARG.
 *  - The first call on a device looks up the scratch address (a host-side
 *    runtime query, done once per device under a lock); make that first call
 *    before any stream capture begins.  A cudaDeviceReset of the device
 *    invalidates the looked-up address: do not call this entry point again in
 *    a process that has reset the device.
 *  - All calls share the one scratch array: calls whose GPU work overlaps
 *    (different streams, contexts or threads without ordering) race on it.
 *    Every entry a call reads is written by that same call first, so nothing
 *    needs clearing between calls. */
idg_status idg_get_moments_noalloc(idg_ctx *ctx, double *out6_dev, void *stream);

/* Absolute residuals ||R_W/Omega||_2 of the iterations since the last
 * (re)start, oldest first; *n receives the count copied (<= cap). */
idg_status idg_get_residual_history(idg_ctx *ctx, double *out, int cap, int *n);

/* Face moment fluxes Phi_f = sum_k w_k psi_k F_k (Eq. 27) of the last
 * iteration, host [nface][4] float64, faces numbered i-faces row by row then
 * j-faces row by row; normal from the lower to the higher cell index side. */
idg_status idg_get_face_flux_moments(idg_ctx *ctx, double *phi4, void *stream);

/* Force (x, y) of the gas on the walls of the sides in side_mask (bit s =
 * side s; each must be IDG_BC_WALL): the sum over their faces of the momentum
 * components of Phi (Eq. 27) of the last iteration, oriented from the gas
 * into the wall (the objective of idg_adjoint).  force2: host, 2 doubles. */
idg_status idg_get_wall_force(idg_ctx *ctx, int side_mask, double *force2, void *stream);

/* Wall quantities of the last iteration on the faces of one wall side, in
 * face order (the face numbering of idg_get_face_flux_moments restricted to
 * that side): the surface pressure, shear stress and heat flux the paper
 * plots along the cylinder wall (Section 3).  With n the unit normal from the
 * gas into the wall, t = (-n_y, n_x), S the face length, (P_x, P_y) = the
 * momentum components of Phi (Eq. 27) oriented along n, over S (the momentum
 * flux into the wall per unit length, Pi n, which is the stress on the wall
 * since the mass flux through it is zero) and E the energy component oriented
 * along n, over S, each face gives five float64:
 *   x, y   the face midpoint,
 *   p      = n . (Pi n)                  normal stress (pressure),
 *   tau_w  = t . (Pi n)                  shear stress,
 *   q_n    = E - U_w . (Pi n)            heat flux into the wall: the energy
 *                                        flux in the frame of the wall,
 *                                        whose velocity U_w is the side's
 *                                        boundary velocity (idg_set_boundary).
 * Nondimensional like every output (rho_ref = 1, velocity unit sqrt(2 RT_ref)).
 * out5: host, room for cap faces (cap 0 and out5 NULL: count only);
 * *nfaces receives the side's face count (rows beyond cap are not written).
 * IDG_ERR_ARG if the side is not a wall. */
idg_status idg_get_wall(idg_ctx *ctx, int side, double *out5, int cap, int *nfaces, void *stream);

/* One iteration with a CUDA event recorded between its kernel launches on
 * the caller's stream (synchronises it).  kernel_ms[0..5] receives the
 * device time of: cell prep, interior faces, boundary faces, macroscopic
 * predictor, forward sweep, backward sweep (0 for a kernel not launched). */
idg_status idg_iterate_profiled(idg_ctx *ctx, void *stream, double *kernel_ms);

/* Launch-shape tuning of the wavefront kernels (after idg_bind_workspace;
 * no effect on results).  IDG_TUNE_SWEEP_TV: discrete velocities per thread
 * block of the micro LU-SGS sweeps (power of two, 1..32, times min(ni, nj)
 * at most 512).  IDG_TUNE_SWEEP_STAGES / IDG_TUNE_MACRO_STAGES: hyperplanes
 * prefetched ahead by the micro / macroscopic sweeps (2, 4 or 8; 2 halves the
 * micro sweeps' shared memory, so more velocity tiles are resident at once
 * on a large velocity grid; the macroscopic sweep takes 2 by default for a
 * float64 block with min(ni, nj) above 213, its records filling shared
 * memory).  Returns
 * IDG_ERR_ARG for a value that is invalid or does not fit in shared memory.
 * IDG_TUNE_SWEEP_VPT: consecutive velocities per thread of the micro sweeps
 * (1, 2 or 4; all instances of a batch must agree).  Any velocity count takes
 * all three: the library stores each cell's velocities rounded up to a
 * multiple of 4, the extra ones being ghost velocities of zero weight at
 * xi = 0 that enter no moment and no flux and never reach the caller.
 * IDG_TUNE_GRAPH (1 default, 0 off): idg_iterate replays chunks of 16
 * iterations (and single iterations) as captured CUDA graphs on a
 * library-owned stream that is ordered after, and before, the caller's
 * stream by events.  IDG_TUNE_MACRO_KIND: the macroscopic LU-SGS sweeps of a
 * structured block (Eq. 30) with one thread per line of cells of the shorter
 * axis (1, default for IDG_MIXED) or with two threads per cell of each i+j
 * hyperplane (0, default for IDG_FP64); setting it re-derives the
 * macroscopic prefetch depth (8 where the records fit in shared memory, else
 * 4, else 2); the same lexicographic dependency order, results equal up to
 * the rounding order of a cell's neighbour sum; all instances of a batch
 * must agree. */
enum { IDG_TUNE_SWEEP_TV = 1, IDG_TUNE_SWEEP_STAGES = 2, IDG_TUNE_MACRO_STAGES = 3, IDG_TUNE_GRAPH = 4,
       IDG_TUNE_SWEEP_VPT = 5, IDG_TUNE_MACRO_KIND = 6 };
idg_status idg_set_tuning(idg_ctx *ctx, int key, int value);
idg_status idg_get_tuning(const idg_ctx *ctx, int key, int *value);

/* Sizes and host-side tables (valid after the corresponding setters). */
idg_status idg_get_sizes(const idg_ctx *ctx, int *ncell, int *nvel, int *nface);
idg_status idg_get_dt(const idg_ctx *ctx, double *dt);
idg_status idg_velocity_grid(const idg_ctx *ctx, double *ux, double *uy, double *w);

/* ---------------------------------------------------------------------------
 * Batches: several bound contexts (same precision and device; sizes, gases,
 * boundaries and tunings may differ) advanced together, each kernel of an
 * iteration launched once over all of them (blocks map to instances through
 * prefix sums), chunks of iterations replayed as CUDA graphs.  An instance
 * stops iterating once its own relative residual is <= tol; the others go
 * on.  Residual histories and states stay in each context (idg_get_*).
 * A context may belong to one batch at a time and must not be iterated on
 * its own while a batch call is running.
 * ------------------------------------------------------------------------- */
typedef struct idg_batch idg_batch;
idg_status idg_batch_create(idg_batch **out, idg_ctx *const *ctxs, int n);
void idg_batch_destroy(idg_batch *b);
const char *idg_batch_last_error(const idg_batch *b);
/* small device workspace for the batch's tables (caller-owned, 256-B aligned) */
idg_status idg_batch_workspace_size(idg_batch *b, size_t *bytes);
idg_status idg_batch_bind_workspace(idg_batch *b, void *dev_ptr, size_t bytes);
/* Up to max_iter iterations of every unconverged instance.  converged (may
 * be NULL): per instance 1 if its relative residual is <= tol.  max_residual:
 * the largest relative residual.  Returns IDG_ERR_NOT_CONVERGED if tol > 0
 * and an instance is left above it, IDG_ERR_NONFINITE if one diverged. */
idg_status idg_batch_iterate(idg_batch *b, int max_iter, double tol, void *stream, int *iters_done,
                             double *max_residual, int *converged);

/* ---------------------------------------------------------------------------
 * Discrete adjoint of the steady solve.  The paper has no adjoint; this one
 * differentiates the discrete iteration of Section 2.3 (Eq. 10-20, 23, 26-32,
 * 34-35) in float64 at the state the context holds, which should be
 * converged (the gradient is that of the steady state only to the extent
 * that it is).  With u = (f~, W) and one iteration u -> u + P^-1 R(u) (macro
 * predictor, then micro LU-SGS), the adjoint iterates the transposed
 * fixed-point map lambda <- dJ/du + (I + P^-1 dR/du)^T lambda: the transposed
 * micro sweeps, then the transposed macroscopic block sweeps (Euler flux
 * Jacobians), then one vector-Jacobian product of the residual through the
 * face fluxes, the reconstruction, the limiter and the cell equilibria.  It
 * converges at the rate of the forward iteration.  At its fixed point
 * dJ/dp = dJ/dp|_u + lambda^T d(iteration)/dp.
 *
 * Objective J: the x (IDG_OBJ_FORCE_X) or y (IDG_OBJ_FORCE_Y) force of the gas
 * on the walls of the sides in side_mask (bit s = side s; each a wall): the sum
 * over their faces of the momentum flux Phi (Eq. 27) through the face,
 * oriented from the gas into the wall.  Lid shear force of a cavity, drag of
 * a body.
 *
 * Parameters (params[i], one gradient each in grad[i]):
 *   IDG_PARAM(IDG_PAR_KN, 0)            the Knudsen number of idg_set_gas
 *   IDG_PARAM(IDG_PAR_WALL_T, mask)     temperature (units of T_ref) of the
 *                                       walls of the sides in mask, together
 *   IDG_PARAM(IDG_PAR_WALL_U, mask)     x velocity of those walls
 *   IDG_PARAM(IDG_PAR_WALL_V, mask)     y velocity of those walls
 *
 * Closed domains (walls and periodic sides only): the mass residuals sum to
 * zero identically, so the steady states form a one-parameter family indexed
 * by the total mass M = sum_c Omega_c rho_c, and the iteration has a neutral
 * mode.  There the adjoint also solves for the total mass as a second
 * right-hand side and returns dJ/dp at fixed M (the mass of the context's
 * state); both solves run together.  With a far-field side the steady state
 * is unique and one solve is run.
 *
 * workspace: caller-owned device memory, 256-byte aligned, at least
 * idg_adjoint_workspace_size bytes, used only during the call.  The context's
 * own workspace and state are read, not changed.  Iterates until the norm of
 * the update of lambda, relative to the first one, is <= tol, or max_iter
 * (1 ... 65536) iterations.  J receives the objective at the context's state;
 * residual the last relative update.  Returns IDG_ERR_ARG for an invalid
 * objective, parameter or side (not a wall), or when numerics flags are set;
 * IDG_ERR_NOT_CONVERGED (results still written) if tol > 0 was not reached;
 * IDG_ERR_NONFINITE if the update overflowed.  Synchronises the stream.
 * ------------------------------------------------------------------------- */
enum { IDG_OBJ_FORCE_X = 0, IDG_OBJ_FORCE_Y = 1 };
enum { IDG_PAR_KN = 0, IDG_PAR_WALL_T = 1, IDG_PAR_WALL_U = 2, IDG_PAR_WALL_V = 3 };
#define IDG_PARAM(kind, side_mask) ((kind) | ((side_mask) << 8))
idg_status idg_adjoint_workspace_size(idg_ctx *ctx, size_t *bytes);
idg_status idg_adjoint(idg_ctx *ctx, int objective, int side_mask, const int *params, int nparam,
                       void *workspace, size_t bytes, int max_iter, double tol, void *stream, double *J,
                       double *grad, int *iters_done, double *residual);
/* Solver of idg_adjoint's linear system (I - M^T) lambda = dJ/du (the
 * paper has no adjoint; a service of the library).  IDG_ADJ_FIXED_POINT
 * (default): the transposed fixed-point iteration lambda <- dJ/du + M^T
 * lambda, which converges at the rate of the forward iteration when the
 * spectral radius of M^T is below one.  IDG_ADJ_GMRES: restarted GMRES(restart)
 * on the same system with one transposed pass per Krylov vector; it needs no
 * bound on the spectral radius (the linearisation, with the limiter frozen
 * at its active branch, can have modes just outside the unit circle where the
 * nonlinear forward iteration still converges), only a domain with a far
 * field (one right-hand side; a closed domain returns IDG_ERR_ARG at
 * idg_adjoint).  restart in [2, 64]; idg_adjoint_workspace_size grows by
 * (restart + 4) float64 vectors of 2 ncell nvel + 4 ncell.  In GMRES mode
 * max_iter counts transposed passes and tol bounds the relative residual
 * ||dJ/du - (I - M^T) lambda|| / ||dJ/du||.  Takes effect at the next
 * idg_adjoint_workspace_size / idg_adjoint. */
enum { IDG_ADJ_FIXED_POINT = 0, IDG_ADJ_GMRES = 1 };
idg_status idg_set_adjoint_solver(idg_ctx *ctx, int method, int restart);
/* How idg_adjoint linearises the Venkatakrishnan limiter (Eq. 16-17).
 * IDG_ADJ_LIMITER_EXACT (default): the factor phi of each (cell, velocity,
 * component) is differentiated with its binding face and extreme neighbour
 * fixed -- the exact derivative of the iteration where it is smooth.  Near a
 * local extremum of a velocity's fb+ field, phi's derivative grows like
 * 1/d (d the extrapolated increment to the binding face), and the exact
 * linearisation can be unstable where the forward iteration is not.
 * IDG_ADJ_LIMITER_FROZEN: phi is held at its value at the linearisation
 * point (its derivative dropped): the gradient of the scheme with phi fixed,
 * an approximation of the exact one.  Takes effect at the next idg_adjoint;
 * IDG_ERR_ARG for another mode. */
enum { IDG_ADJ_LIMITER_EXACT = 0, IDG_ADJ_LIMITER_FROZEN = 1 };
idg_status idg_set_adjoint_limiter(idg_ctx *ctx, int mode);
/* The adjoint variables lambda = (lambda_G, lambda_H [ncell][nvel], lambda_W
 * [ncell][4]) left in the workspace by the last idg_adjoint call of this
 * context.  which = 0: the adjoint of the returned gradient (for a closed
 * domain, the fixed-mass combination of the two solves); 1: the solve seeded
 * by the objective alone; 2: the one seeded by the total mass (closed domains
 * only).  Host arrays; any may be NULL. */
idg_status idg_adjoint_state(idg_ctx *ctx, const void *workspace, int which, double *lamG, double *lamH,
                             double *lamW, void *stream);

#ifdef __cplusplus
}
#endif
#endif
