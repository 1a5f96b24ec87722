/*
 * m2c.h -- C ABI of libm2cgpu.so, a GB300 (sm_103a) solver for the
 * multi-material compressible flow step of M2C (arXiv 2508.16387).
 *
 * One call to m2c_step advances a Cartesian grid by whole time steps of the
 * method of the paper's Sec. 4: cell-centred finite volumes (Sec. 4.2, Eq.
 * NS_discretized with the viscous and source terms off), MUSCL reconstruction
 * of the primitive variables with the modified van Albada limiter (App. D),
 * the HLLC flux (App. C.4) on faces between cells of one material, the FIVER
 * flux on faces where the level set changes sign (Sec. 4.2, exact
 * two-material Riemann problem, Eq. 1DRiemannProblem), the second-order TVD
 * Runge-Kutta scheme (Sec. 4.3), level-set advection (Sec. 3.5.1, Eq.
 * levelset; third-order upwind finite differences, Sec. 4.4), periodic
 * reinitialisation (Eq. reinit) and the phase update of Sec. 2.3 step (6).
 *
 * Conventions. SI units. A grid has nx*ny*nz cells of edge h; arrays are
 * structure-of-arrays with x fastest: field f of cell (i,j,k) is at
 * a[f*N + (k*ny + j)*nx + i], N = nx*ny*nz. The conserved state is
 * W = (rho, rho u, rho v, rho w, rho E), E = e + |V|^2/2; primitive arrays are
 * (rho, u, v, w, p). Material 1 is where phi < 0, material 0 elsewhere.
 *
 * Memory ownership. The caller owns all memory. Device arrays passed to the
 * library are borrowed for the life of the context (or of the call, for the
 * one-shot entry points); the library allocates no device memory. All solver
 * scratch lives in one caller-provided device workspace of
 * m2c_workspace_bytes() bytes, 256-byte aligned; the one-shot Riemann and
 * shock-state calls stage host arrays through a caller-provided workspace of
 * m2c_riemann_workspace_bytes() bytes.
 *
 * Errors. Every entry point returns an m2c_status; no exception crosses the
 * ABI. Launches are asynchronous on the context's stream; errors raised on
 * the device (non-physical state, Riemann non-convergence, list overflow) are
 * latched in the workspace and returned by m2c_sync together with the first
 * offending cell. m2c_last_error() gives a text for the last error of a
 * context (NULL: of the last failed call without a context on this thread).
 * Functions are not thread-safe on one context.
 */
#ifndef M2C_H
#define M2C_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  M2C_OK = 0,
  M2C_EINVAL = 1,    /* bad argument */
  M2C_ENOMEM = 2,    /* workspace too small */
  M2C_ECUDA = 3,     /* CUDA runtime error */
  M2C_ENOCONV = 4,   /* Newton / bisection cap reached in the Riemann solver */
  M2C_ENONPHYS = 5,  /* rho <= 0, c^2 <= 0, or a state outside the EOS domain */
  M2C_EVACUUM = 6,   /* the Riemann problem has a vacuum solution (not built) */
  M2C_ETIMEOUT = 7,  /* a bounded device wait ran out */
  M2C_EOVERFLOW = 8  /* an interface work list exceeded its capacity */
} m2c_status;

/* Equations of state (Sec. 3.3 and App. B).
 * M2C_EOS_SG: stiffened gas, NASG with b = e_c = 0: p = (gamma-1) rho e - gamma p_c;
 *   params = {gamma, p_c}; p_c = 0 is a perfect gas.
 * M2C_EOS_MG: Mie-Grueneisen (App. B.3): p = p_R(eta) + rho0 Gamma0 (e - e_R(eta)),
 *   eta = 1 - rho0/rho; params = {rho0, c0, s, Gamma0, e0, eta_min}; eta_min = -inf
 *   (or fewer than 6 params) turns the tensile cutoff off.
 * M2C_EOS_NASG: Noble-Abel stiffened gas (Sec. 3.3, Eq. NASG_EOS):
 *   p = (gamma-1) rho (e - e_c)/(1 - rho b) - gamma p_c, defined for rho b < 1;
 *   params = {gamma, p_c, b, e_c}.
 * M2C_EOS_JWL: Jones-Wilkins-Lee (App. B.2, Eq. JWL_EOS):
 *   p = omega rho e + sum_i A_i (1 - omega rho/(R_i rho0)) exp(-R_i rho0/rho) (the first
 *   exponential, printed with a plus sign, is read with the minus sign of the second);
 *   params = {omega, A1, A2, R1, R2, rho0}.
 * A grid with a NASG or JWL material runs the general bulk kernel (8-row tiles). */
typedef enum { M2C_EOS_SG = 0, M2C_EOS_MG = 1, M2C_EOS_NASG = 2, M2C_EOS_JWL = 3 } m2c_eos_type;

/* M2C_FP64: every operation in FP64. M2C_MIXED: reconstruction, HLLC, the
 * level-set residual and the reinitialisation update in FP32; the pressure
 * from the conserved state, the Runge-Kutta accumulation of W and phi, the
 * level-set values and the exact Riemann solver's Newton iteration in FP64
 * (m2c_set_riemann_start offers an FP32 start for the latter). */
typedef enum { M2C_FP64 = 0, M2C_MIXED = 1 } m2c_precision;

/* Boundary conditions per side (x-, x+, y-, y+, z-, z+): transmissive
 * (zero-gradient ghost values), periodic (both sides of an axis), or symmetry
 * (a mirror plane: the ghost cells are the mirror images of the cells inside,
 * with the velocity component normal to the side negated; the axis of the
 * spherical and cylindrical forms of Sec. 3.4 and the mirror planes of a
 * symmetric problem; needs at least 2 cells along the axis). */
typedef enum { M2C_BC_TRANSMISSIVE = 0, M2C_BC_PERIODIC = 1, M2C_BC_SYMMETRY = 2 } m2c_bc;

typedef struct {
  int type;          /* m2c_eos_type */
  double params[6];
} m2c_eos_desc;

typedef struct m2c_ctx m2c_ctx;

/* Counters of the last completed step, read by m2c_get_stats after m2c_sync. */
typedef struct {
  long interface_faces;  /* faces with different materials, stage 1 of the last step */
  long interface_cells;  /* cells with at least one such face, stage 1 */
  long flipped_cells;    /* cells that changed material in the last step */
  double dt;             /* time step of the next step */
} m2c_stats;

/* Workspace bytes for an nx*ny*nz grid (host arithmetic only; 0 if a size is
 * below 1). The workspace holds what one time step of Sec. 2.3 steps (1)-(6)
 * needs besides the state: the stage state W(1), phi(1) of the Runge-Kutta
 * scheme (Sec. 4.3), the reinitialisation scratch (Eq. reinit), one byte of
 * material flags per cell, the interface work lists of the FIVER flux
 * (Sec. 4.2) and the star pressure of each face's last exact Riemann solve (the
 * start of the next one, FP64); about 120 bytes per cell. */
size_t m2c_workspace_bytes(int nx, int ny, int nz, int precision);

/* Creates a context on the calling thread's current CUDA device for a
 * uniform Cartesian mesh of nx*ny*nz cells of edge h (the finite-volume mesh of
 * Sec. 4.1 with cell-centred control volumes; boundary conditions of Sec. 2.3).
 * At least one
 * axis must have more than one cell, and nx*ny*nz < 2^31 (M2C_EINVAL otherwise).
 * lo: lower corner (only used to report coordinates), h > 0: cell edge,
 * bc[6]: m2c_bc per side, workspace: device pointer of ws_bytes >=
 * m2c_workspace_bytes(), stream: a cudaStream_t (NULL = legacy default stream).
 * Defaults: CFL 0.5, reinitialisation every 10 steps with 5 iterations.
 * Argument errors return before any device work; they and a failed first
 * device call (M2C_ECUDA, no context created) leave the reason in
 * m2c_last_error(NULL). */
m2c_status m2c_init_grid(m2c_ctx** out, int nx, int ny, int nz, const double lo[3], double h, const int bc[6],
                         int precision, void* workspace, size_t ws_bytes, void* stream);

/* Material 0 (phi >= 0) or 1 (phi < 0) gets an EOS (Sec. 3.3, App. B.1-B.3):
 * M2C_EOS_SG (gamma > 1, p_c), M2C_EOS_MG (rho0 > 0, c0 > 0, s > 1,
 * Gamma0 > 0 [, e0 [, eta_min]]), M2C_EOS_NASG (gamma > 1, p_c, b >= 0, e_c)
 * or M2C_EOS_JWL (omega > 0, A1, A2, R1 > 0, R2 > 0, rho0 > 0); anything else
 * is M2C_EINVAL. */
m2c_status m2c_set_eos(m2c_ctx* ctx, int material, int type, const double* params, int nparams);

/* CFL number of dt = CFL h / max_cells sum_d (|V_d| + c) (the sum runs over the
 * axes with more than one cell), and the reinitialisation schedule: after every
 * reinit_every-th step, reinit_iters pseudo-time iterations (0 disables). */
m2c_status m2c_set_scheme(m2c_ctx* ctx, double cfl, int reinit_every, int reinit_iters);

/* Scheme options beyond the default of m2c_init_grid (TVD RK2, the modified van
 * Albada limiter, HLLC, the CFL time step): the paper's other choices.
 *  rk: Runge-Kutta scheme of Sec. 4.3: 2 = TVD RK2 (default), 3 = TVD RK3
 *      (W2 = 3/4 W + 1/4 W1 + 1/4 dt R(W1), W' = 1/3 W + 2/3 W2 + 2/3 dt R(W2);
 *      its second stage state needs the workspace of m2c_workspace_bytes_rk(.., 3),
 *      M2C_ENOMEM if the context's workspace is smaller), 1 = forward Euler.
 *  limiter: M2C_LIM_VAN_ALBADA (App. D, the modified limiter) or M2C_LIM_MC
 *      (App. D, Eq. theta: phi = max(0, min(alpha theta, (1 + theta)/2, alpha)),
 *      alpha = mc_alpha, 1 <= alpha <= 2).
 *  flux: M2C_FLUX_HLLC (App. C.4) or M2C_FLUX_LLF (App. C.1, Eq.
 *      Lax-Friedrichs: the local Lax-Friedrichs flux with the largest |u_n| + c of
 *      the two face states); the FIVER flux of an interface face uses it too.
 *  dt_fixed: > 0 = a constant time step instead of the CFL rule (Sec. 4.3).
 *  geom: M2C_GEOM_CARTESIAN (default), or the reduced forms of Sec. 3.4 in
 *      which the grid's x axis is the radius r, r_i = x0 + (i + 1/2) h:
 *      M2C_GEOM_SPHERICAL (Eq. euler1d_spherical; ny = nz = 1) or
 *      M2C_GEOM_CYLINDRICAL (Eq. Euler_cylindrical; ny = 1, z the axial
 *      coordinate). The geometric source S = -(alpha/r) u_r (rho, rho u, rho v,
 *      rho w, rho E + p), alpha = 2 or 1, is evaluated at the cell centre from
 *      the stage state and added to the residual after the flux sum; the
 *      level-set equation keeps its Cartesian form. A symmetry side at r = 0
 *      (x0 = 0) is the axis or centre. x0 >= 0.
 *  band_beta, band_gamma: the narrow-band level set of Sec. 4.4 (the local
 *      level set of Peng et al., J. Comput. Phys. 155, 1999), tube radii in
 *      cells, 0 < band_beta < band_gamma; band_gamma = 0 (default) solves the
 *      level-set equation in the whole domain. The advection velocity is scaled
 *      by c = 1 for |phi| <= beta, (|phi| - gamma)^2 (2|phi| + gamma - 3 beta)/
 *      (gamma - beta)^3 between the radii and 0 beyond; after the Runge-Kutta
 *      update and the scheduled reinitialisation phi is clipped to
 *      [-gamma, gamma].
 * Any non-default option, and any symmetry side, selects the general
 * instantiation of the bulk kernel (8-row tiles). M2C_EINVAL for a value
 * outside these sets. */
typedef enum { M2C_LIM_VAN_ALBADA = 0, M2C_LIM_MC = 1 } m2c_limiter;
typedef enum { M2C_FLUX_HLLC = 0, M2C_FLUX_LLF = 1 } m2c_flux;
typedef enum { M2C_GEOM_CARTESIAN = 0, M2C_GEOM_CYLINDRICAL = 1, M2C_GEOM_SPHERICAL = 2 } m2c_geom;
typedef struct {
  int rk;
  int limiter;
  int flux;
  double mc_alpha;
  double dt_fixed;
  int geom;
  double x0;
  double band_beta;
  double band_gamma;
} m2c_options;
m2c_status m2c_set_options(m2c_ctx* ctx, const m2c_options* opt);

/* Workspace bytes for an nx*ny*nz grid stepped with the Runge-Kutta scheme of
 * order rk (Sec. 4.3): rk = 1 or 2 as m2c_workspace_bytes, rk = 3 adds the
 * second stage state (48 bytes per cell). The RK2 layout is a prefix of it. */
size_t m2c_workspace_bytes_rk(int nx, int ny, int nz, int precision, int rk);

/* M2C_MIXED grids only (M2C_EINVAL otherwise for fp32_start = 1). fp32_start
 * = 0 (default): the FIVER kernel runs the FP64 Newton iteration of
 * m2c_solve_riemann. fp32_start = 1: it starts the iteration on FP32 wave
 * curves and finishes with FP64 Newton steps, as m2c_solve_riemann_mixed
 * (an option beyond the paper's method, which does not discuss precision). */
m2c_status m2c_set_riemann_start(m2c_ctx* ctx, int fp32_start);

/* Tile of the bulk stage kernel: 32 x tile_rows (4 or 8; 16 for M2C_MIXED)
 * columns marching tile_z cells along z (0: automatic). M2C_FP64 results do
 * not depend on the tiling (bitwise); M2C_MIXED results agree to FP32 rounding
 * (FP32 multiply-adds may be contracted differently in the code that opens a
 * z-chunk and in the kernels of other tile heights). Default: 16 rows for
 * M2C_MIXED grids large enough to give every SM 8 tiles of 16 rows and 16
 * planes, else 8. */
m2c_status m2c_set_tiling(m2c_ctx* ctx, int tile_rows, int tile_z);

/* Borrows the device arrays W (5N doubles, the conserved state of Sec. 3.2,
 * Eq. NSEquation_terms) and phi (N doubles, the level set of Sec. 3.5.1 whose
 * sign gives the material) as the state, and sets time t and step counter
 * step; the first time step (Sec. 4.3) is reduced at the next m2c_step. The
 * arrays stay the caller's and are updated in place by m2c_step. The FIVER
 * solves start each face's Newton iteration from that face's star pressure of
 * its previous solve; a new state clears those starts, so a run restarted from
 * its (W, phi, t, step) agrees with the uninterrupted run to rounding (the same
 * roots within the iteration's tolerance), not bit for bit. M2C_EINVAL if an
 * array is NULL or an EOS has not been set. */
m2c_status m2c_set_state(m2c_ctx* ctx, double* W, double* phi, double t, long step);

/* Fills the borrowed W from device primitive arrays prims (5N: rho, u, v, w, p)
 * using the EOS of each cell's material (from the sign of phi). */
m2c_status m2c_prims_to_state(m2c_ctx* ctx, const double* prims);

/* The inverse: primitive fields (rho, u, v, w, p) of the current state into
 * the device array prims (5N doubles, SoA, x fastest, caller-owned), FP64
 * with each cell's material EOS (material 1 where phi < 0; Sec. 3.3).
 * Asynchronous on the context's stream; a non-physical cell is latched
 * (M2C_ENONPHYS from m2c_sync) and its entries are unspecified. */
m2c_status m2c_state_to_prims(m2c_ctx* ctx, double* prims);

/* Copies host arrays into / out of the borrowed state (pinned host memory gives
 * asynchronous copies; m2c_download_state synchronises the stream). */
m2c_status m2c_upload_state(m2c_ctx* ctx, const double* W_host, const double* phi_host);
m2c_status m2c_download_state(m2c_ctx* ctx, double* W_host, double* phi_host);

/* Advances nsteps time steps (m2c_step) from the state in the host arrays
 * W_host (5N doubles) and phi_host (N doubles), the layout of m2c_set_state, and
 * writes the new state back into them: the upload, the steps and the download
 * of the host-resident time-stepping loop in one call, asynchronous on the
 * context's stream (m2c_sync waits; the host arrays must not be touched before).
 * The copies go one state component at a time: when a call uses the same host
 * arrays as the previous call, it uploads each component on a second stream as
 * soon as the previous call's download of that component has finished, so the
 * two directions of the host link overlap. Host arrays in pinned memory are
 * required for the copies to be asynchronous. The time step is recomputed from
 * the uploaded state (as after m2c_upload_state). Errors: M2C_EINVAL (null
 * arguments, nsteps < 0, no state), M2C_ECUDA. */
m2c_status m2c_step_host(m2c_ctx* ctx, double* W_host, double* phi_host, int nsteps);

/* Enqueues nsteps time steps on the context's stream. One step is Sec. 2.3
 * steps (1)-(6) with the fluid and level-set updates of the TVD Runge-Kutta
 * scheme (Sec. 4.3): the time step from the CFL number, two stages of the
 * residual of Sec. 4.2 (Eq. NS_discretized) and of the level-set equation
 * (Eq. levelset), the scheduled reinitialisation (Eq. reinit) and the phase
 * update. Asynchronous; device errors are read by m2c_sync. */
m2c_status m2c_step(m2c_ctx* ctx, int nsteps);

/* Batches: several contexts of one precision stepped together, one launch per
 * kernel for all of them (the bulk kernel takes its tiles from all grids of
 * the batch, largest grid first; every grid keeps its own time step, error
 * latch, work lists and reinitialisation schedule, counted from its own step).
 * workspace: caller's device buffer of m2c_batch_workspace_bytes(k) bytes,
 * 256-byte aligned, borrowed for the life of the batch. tuning (may be NULL) =
 * {tile rows 4, 8 or (mixed) 16, tile length along z (0: automatic), schedule (0: fixed
 * stride over tiles, 1: atomic tile counter), blocks per SM of a persistent
 * grid (0: one block per tile)}. m2c_batch_create synchronises (it uploads the
 * descriptors and reduces the first time steps). */
typedef struct m2c_batch m2c_batch;
size_t m2c_batch_workspace_bytes(int k);
m2c_status m2c_batch_create(m2c_batch** out, m2c_ctx** ctxs, int k, void* workspace, size_t bytes,
                            const int tuning[4]);

/* Enqueues nsteps steps of the batch on the first context's stream (no host
 * synchronisation). */
m2c_status m2c_batch_step(m2c_batch* b, int nsteps);

/* Captures nsteps steps of the batch into a CUDA graph (instantiated, returned
 * as an opaque cudaGraphExec_t); m2c_batch_launch_graph launches it on the
 * batch's stream (any number of times: every grid reads its own step counter on
 * the device) and advances the step counters; m2c_graph_destroy frees it. */
m2c_status m2c_batch_capture(m2c_batch* b, int nsteps, void** graph_exec);
m2c_status m2c_batch_launch_graph(m2c_batch* b, void* graph_exec);
void m2c_graph_destroy(void* graph_exec);
void m2c_batch_destroy(m2c_batch* b);

/* Writes the residual of one Runge-Kutta stage of the current state, without
 * advancing it: R (5N) = dW/dt and L (N) = dphi/dt, device arrays. */
m2c_status m2c_residual(m2c_ctx* ctx, double* R, double* L);

/* Blocks until the stream is idle; returns the first latched device error,
 * the time, the step counter and the offending cell (-1 if none). Any of the
 * output pointers may be NULL. Clears the latched error. The paper's solver
 * checks state admissibility (rho > 0, c^2 > 0, the EOS domain of App. B) and
 * Riemann-solver convergence (Sec. 4.2) on the host; here those checks run
 * on the device and are reported by this call. */
m2c_status m2c_sync(m2c_ctx* ctx, double* t, long* steps, long* err_cell);

m2c_status m2c_get_stats(m2c_ctx* ctx, m2c_stats* out);

/* Device bytes a host-array call of m2c_solve_riemann, m2c_solve_riemann_mixed
 * (n problems) or m2c_shock_state (n = 1) stages its arrays through. */
size_t m2c_riemann_workspace_bytes(int n);

/* Batch of n exact two-material Riemann problems (Sec. 4.2, Eq.
 * 1DRiemannProblem). L and R are SoA (rho[n], u[n], p[n]); out is SoA
 * (p*[n], u*[n], rho*_L[n], rho*_R[n]); iters[n] and status[n] (may be NULL)
 * get the iteration count and per-problem m2c_status. on_device = 1: all
 * arrays are device pointers, workspace is unused (may be NULL) and the call
 * is asynchronous on stream; 0: host arrays, staged through the caller's
 * device workspace (256-byte aligned, ws_bytes >= m2c_riemann_workspace_bytes(n);
 * M2C_ENOMEM if smaller), and the call blocks. Returns the first non-OK
 * status of the batch (host arrays) or M2C_OK (device arrays; read status[]).
 * M2C_EINVAL, before any device work and with the reason in
 * m2c_last_error(NULL): n < 0, a NULL array or descriptor, or EOS parameters
 * that m2c_set_eos rejects. */
m2c_status m2c_solve_riemann(int n, const m2c_eos_desc* eosL, const double* L, const m2c_eos_desc* eosR,
                             const double* R, double* out, int* iters, int* status, int on_device, void* workspace,
                             size_t ws_bytes, void* stream);

/* The same batch solved the way the FIVER kernel of the M2C_MIXED path solves
 * it (Sec. 4.2 with the mixed-precision reading): Newton iterations on FP32
 * wave curves from the same start, then one FP64 Newton step on the FP64 wave
 * curves (two when the first moves p by more than 1e-9 |p|); u* and the star
 * densities follow to first order in the last step. Problems whose FP32
 * iteration fails, signals a vacuum or ends more than 1e-5 |p| from the FP64
 * step are solved by the FP64 iteration of m2c_solve_riemann. iters counts
 * the FP32 and FP64 steps. Arguments, layout, ownership and errors as for
 * m2c_solve_riemann. */
m2c_status m2c_solve_riemann_mixed(int n, const m2c_eos_desc* eosL, const double* L, const m2c_eos_desc* eosR,
                                   const double* R, double* out, int* iters, int* status, int on_device,
                                   void* workspace, size_t ws_bytes, void* stream);

/* Post-shock state of a shock moving in +x into the state w = (rho, u, p) with
 * pressure p1 behind it (the right-facing wave of the exact Riemann solver of
 * Sec. 4.2; the Rankine-Hugoniot state of a planar shock): out = (rho1, u1,
 * shock speed). Host arrays w and out; the result passes through the caller's
 * device workspace (256-byte aligned, >= m2c_riemann_workspace_bytes(1)
 * bytes); enqueued on stream, then blocks. M2C_EINVAL as for
 * m2c_solve_riemann, and for p1 <= p. */
m2c_status m2c_shock_state(const m2c_eos_desc* eos, const double w[3], double p1, double out[3], void* workspace,
                           size_t ws_bytes, void* stream);

/* Allocation-free stage residual. The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory, such as a host
 * application whose device memory comes from its own fixed pool, or code that
 * must not trigger the device-wide synchronisation of cudaMalloc and cudaFree.
 * It computes what m2c_residual computes (R = dW/dt, 5N doubles, and L =
 * dphi/dt, N doubles, device arrays) for the state W (5N) and phi (N) on an
 * nx*ny*nz grid with the given EOS of material 0 (phi >= 0) and 1 (phi < 0),
 * with no context and no workspace. Its scratch is one file-scope device array
 * of m2c_residual_noalloc_scratch_bytes() bytes (about 10.5 MB), held by every
 * GPU that loads the library until the process exits. Limits and behaviour:
 *  - nx*ny*nz <= M2C_NOALLOC_MAX_CELLS (262144, e.g. 64^3); larger grids, and
 *    grids, boundary conditions or EOS that m2c_init_grid or m2c_set_eos would
 *    reject, are rejected with M2C_EINVAL before any launch, and
 *    m2c_last_error(NULL) says why.
 *  - each device that calls it gets its own set-up (the array's address, the
 *    kernels' shared-memory limits); calls on several devices are allowed.
 *  - the first call on a device looks up the array's device address with that
 *    device current.
 *  - every call shares the one array: calls whose work overlaps on the GPU
 *    (two streams, two host threads) race; serialise them. Each call clears
 *    the counters it needs and synchronises the stream before returning, so
 *    errors raised on the device are returned by the call itself.
 *  - it calls no cudaMalloc, cudaFree or allocating library routine. */
#define M2C_NOALLOC_MAX_CELLS 262144
size_t m2c_residual_noalloc_scratch_bytes(void);
m2c_status m2c_residual_noalloc(int nx, int ny, int nz, double h, const int bc[6], const m2c_eos_desc* eos0,
                                const m2c_eos_desc* eos1, int precision, const double* W, const double* phi,
                                double* R, double* L, void* stream);

/* Kernel timing: while enabled (enable = 1), m2c_step records a CUDA event
 * pair on the context's stream around every kernel launch; enable = 2 records
 * them around the bulk stage kernel only (least overhead on the step);
 * 0 stops. m2c_profile_read synchronises
 * the stream, returns the summed event time (ms) and the number of launches of
 * the bulk stage kernel, and starts a new count; m2c_profile_read_kernels does
 * the same for every kernel kind: [0] bulk stage, [1] FIVER, [2] interface-cell
 * finish, [3] reinitialisation, [4] phase update, [5] end of step. */
m2c_status m2c_profile(m2c_ctx* ctx, int enable);
m2c_status m2c_profile_read(m2c_ctx* ctx, double* total_ms, long* launches);
m2c_status m2c_profile_read_kernels(m2c_ctx* ctx, double ms[6], long launches[6]);

/* Releases a context (host memory of the library only; the borrowed state
 * and workspace stay with the caller and may be freed after the context's
 * stream is idle). The paper has no counterpart: this is resource ownership
 * of the C ABI. */
void m2c_destroy(m2c_ctx* ctx);

/* Text of the last error of a context; with NULL, of the last failed call on
 * this thread that has no context (m2c_init_grid before a context exists,
 * m2c_solve_riemann, m2c_solve_riemann_mixed, m2c_shock_state,
 * m2c_residual_noalloc). */
const char* m2c_last_error(const m2c_ctx* ctx);
const char* m2c_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* M2C_H */
