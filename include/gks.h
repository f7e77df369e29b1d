/*
 * gks.h -- C ABI of libgks: one two-stage time step of the third-order
 * compact gas-kinetic scheme with two-step multi-resolution WENO
 * reconstruction on tetrahedral meshes, on one NVIDIA GB300 (sm_103a).
 *
 * Method (paper: Ji, Zhao, Shyy, Xu, "Two-step multi-resolution
 * reconstruction-based compact gas-kinetic scheme on tetrahedral mesh"):
 *   - cell averages W and cell-averaged gradients dW are the unknowns (Sec. 2.3);
 *   - each stage reconstructs a quadratic R per cell and component from the
 *     compact stencil (Sec. 4.1-4.3), evaluates the time-dependent kinetic
 *     solution at the three Gauss points of every face (Sec. 2.2, Sec. 4.5),
 *     and updates W by the face fluxes and dW by the divergence theorem
 *     applied to the time-accurate interface values (Sec. 2.3, Sec. 3);
 *   - two stages form one fourth-order step (Sec. 3, Eq. s2o4).
 *
 * Conventions shared by every entry point:
 *   - Return value: GKS_OK (0) or a negative gks_status; gks_last_error()
 *     then returns a message (thread-local, valid until the next call on
 *     the same thread).  No C++ exception crosses this interface.
 *   - Host arrays are row-major and are copied; the caller keeps ownership.
 *   - Device pointers (prefix d_) must be device memory of the current
 *     device; the caller owns them.  The library never allocates or frees
 *     device memory: all device storage lives in one caller-allocated
 *     workspace of gks_workspace_bytes() bytes.
 *   - State layout: W[5][nc] conservative variables (rho, rho U1, rho U2,
 *     rho U3, rho E); dW[15][nc] with row 3*q + i holding d W_q / d x_i.
 *   - All device work is enqueued on the stream given to gks_state_create;
 *     calls that return host values synchronise that stream.
 *   - Asynchronous CUDA errors and device-side error flags (non-positive
 *     density or pressure in an updated cell average) surface at the next
 *     gks_step / gks_get_state / gks_sync as GKS_E_CUDA / GKS_E_STATE.
 */
#ifndef GKS_H
#define GKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t gks_status;
enum {
    GKS_OK = 0,
    GKS_E_ARG = -1,         /* invalid argument (null pointer, bad size, bad option) */
    GKS_E_MESH = -2,        /* invalid mesh (id out of range, non-positive volume,
                               face shared by more than two cells, ...) */
    GKS_E_STENCIL = -3,     /* stencils not built, or a cell's least-squares system
                               is singular (count in gks_stencil_build's output) */
    GKS_E_STATE = -4,       /* non-positive density or pressure in a cell average */
    GKS_E_CUDA = -5,        /* a CUDA runtime call failed */
    GKS_E_TIMEOUT = -6,     /* reserved: a bounded device wait gave up */
    GKS_E_NOMEM = -7,       /* host allocation failed or workspace too small */
    GKS_E_UNSUPPORTED = -8  /* option combination not implemented */
};

/* Scheme parameters (plain data, passed by pointer and copied). */
typedef struct gks_params {
    double gamma;        /* specific heat ratio; K = (5 - 3 gamma)/(gamma - 1), Sec. 2 */
    double cfl;          /* C_CFL of the time-step rule, Sec. 5 Eq. time-step */
    double mu;           /* dynamic viscosity (used when viscous = 1) */
    double eps_weno;     /* epsilon of the nonlinear weights, Sec. 4.2 (paper: 1e-8) */
    double tau_eps;      /* epsilon of the numerical collision time, Sec. 2.2 (0.01) */
    double tau_c;        /* C of the numerical collision time, Sec. 2.2 (1) */
    double prandtl;      /* Prandtl number of the viscous solver (BGK gives 1; other
                            values correct the heat flux, Pr fix below); 1 default */
    double wall_temperature; /* T = p / rho of GKS_BC_ISOTHERMAL_WALL faces; 1 default */
    double wall_velocity[3]; /* velocity of GKS_BC_MOVING_WALL faces (global frame, along
                                the walls); 0 default */
    int32_t weno;        /* 0: linear weights, R = P2 (or P1 at order 2; at order 3 a
                            boundary cell takes the least-squares first-order fit to
                            its P2 stencil's data, Sec. 4.4); 1: nonlinear */
    int32_t order;       /* 3: R^3rd (Eq. final_weno_expression-3rd); 2: R^2nd */
    int32_t smooth_flux; /* 0: full solver Eq. 2nd-flux; 1: smooth Eq. 2nd-smooth-flux */
    int32_t viscous;     /* 0: Euler, tau = 0; 1: tau = mu / p (Sec. 2.2) */
    int32_t precision;   /* 0: FP64 throughout; 1: FP32 bulk (reconstruction, flux,
                            face records and stage states in FP32; FP64 master cell
                            averages updated by compensated sums; cell averages
                            kept as FP32 hi + lo pairs, and the stage-1 face
                            records relative to the mean of the face's two
                            averages, with its flux in FP64); 2: FP32 bulk as 1
                            with the stencil operators M1, M2, the cell moments
                            and their products in the reconstruction in FP64 */
    int32_t wall_constraint; /* 1: at non-slip adiabatic walls (GKS_BC_NOSLIP_WALL) the
                            momenta of the wall cells are reconstructed by the
                            constrained least squares of Sec. 4.4: the step-1 P1
                            vanishes at each wall face's centroid, the step-2 P2 at
                            its three Gauss points (density and energy keep the
                            one-sided stencil); 0 (default): the one-sided stencil
                            for every component.  FP32 and FP64 alike; the adjoint
                            step rejects a state that uses it (GKS_E_UNSUPPORTED) */
} gks_params;

/* Fills the paper's defaults: gamma 1.4, cfl 1, mu 0, eps_weno 1e-8,
 * tau_eps 0.01, tau_c 1, prandtl 1, weno 1, order 3, full flux, Euler, FP64.
 *
 * Pr fix (viscous = 1, prandtl != 1): the BGK model fixes Pr = 1 (Sec. 2);
 * the energy entries of the time-integrated flux get (1/Pr - 1) q, with q
 * the time integral of the heat flux (1/2) int (u1 - U1) |u - U|^2 f dXi of
 * the interface distribution of Eq. 2nd-flux (xi included), U the velocity
 * of the interface equilibrium state in the face frame.  The paper names
 * no formula; this is the correction of the gas-kinetic literature it cites
 * for the Navier-Stokes solver; gks_adjoint_step differentiates it. */
void gks_params_default(gks_params* p);

typedef struct gks_mesh gks_mesh;   /* opaque, library-owned host object */
typedef struct gks_state gks_state; /* opaque, library-owned handle over a
                                       caller-allocated device workspace */

/* ---------------------------------------------------------------- mesh -- */

/* Tetrahedral mesh from vertices and connectivity (Sec. 2.1: cells with four
 * triangular faces).
 *   xyz[n_vert][3]     vertex coordinates
 *   tet[n_cell][4]     vertex ids, positive orientation required
 *   shift[n_cell][4][3] periodic image of each tet vertex: its position is
 *                      xyz[v] + shift * period (NULL: all zero)
 *   period[3]          period per axis, 0 on a non-periodic axis (NULL: none)
 * Faces are the vertex triples, matched across periodic images; a face met
 * once is an open boundary face.  Canonical numbering: faces sorted by their
 * ascending vertex-id triple, then by the image shifts of the second and
 * third vertex relative to the first; each face's unit normal has its first
 * nonzero component positive and points out of its "left" cell.
 * Errors: GKS_E_ARG (null/size), GKS_E_MESH (see enum). */
gks_status gks_mesh_create(const double* xyz, int64_t n_vert, const int64_t* tet,
                           const int8_t* shift, int64_t n_cell, const double* period,
                           gks_mesh** out);
void gks_mesh_destroy(gks_mesh* mesh);

/* A batch of independent cases as one mesh (the disjoint union of their
 * tetrahedra), each case with its own periods and its own time step and
 * time (the time-step rule's minimum is taken per case).
 *   tet_case[n_cell]  case id of each tetrahedron, ascending (cells grouped
 *                     by case); NULL only when n_case == 1
 *   period[n_case][3] periods of each case (NULL: none)
 * Cells of different cases may not share a face (GKS_E_MESH).  Other
 * arguments and the numbering rules as gks_mesh_create, which is the
 * n_case = 1 case of this call. */
gks_status gks_mesh_create_cases(const double* xyz, int64_t n_vert, const int64_t* tet,
                                 const int8_t* shift, int64_t n_cell, const int32_t* tet_case,
                                 int32_t n_case, const double* period, gks_mesh** out);

/* Boundary conditions of the boundary faces (faces with one cell):
 *   GKS_BC_OPEN       ghost side = the interior cell's average with zero
 *                     gradient (outflow by zeroth-order extrapolation; the
 *                     default)
 *   GKS_BC_SLIP_WALL  Sec. 4.4 slip wall: at each Gauss point the ghost is
 *                     the mirror image of the interior reconstruction in the
 *                     face frame (normal momentum reversed; normal derivatives
 *                     reversed except that of the normal momentum; tangential
 *                     derivatives of the normal momentum reversed)
 *   GKS_BC_FIXED      a prescribed state carried past the boundary (the
 *                     Shu-Osher right end of Sec. 5.2; a far field): the
 *                     ghost at each Gauss point is the interior cell's fixed
 *                     state, its average plus its gradient times the offset
 *                     from the centroid, with that gradient.  The fixed state
 *                     is the state given to gks_init_state (or gks_step_host)
 *                     and holds until the next such call, unless
 *                     gks_set_fixed_state has set it: then it holds through
 *                     every later initialisation; a mesh with fixed
 *                     faces needs 20 more working-precision reals a cell of
 *                     workspace.
 *   GKS_BC_NOSLIP_WALL Sec. 4.4 non-slip adiabatic wall at rest: the ghost
 *                     keeps rho and rho E and reverses the three momenta at
 *                     each Gauss point; all derivatives of the momenta are
 *                     kept, all derivatives of rho and rho E reversed
 *                     (impermeable, no heat flux; the wall shear comes from
 *                     the viscous solver, params.viscous = 1)
 *   GKS_BC_ISOTHERMAL_WALL Sec. 4.4 non-slip isothermal wall at rest: the
 *                     ghost has the interior pressure, the reversed velocity
 *                     and the temperature 2 T_w - T (T = p / rho,
 *                     params.wall_temperature = T_w); the derivatives of the
 *                     velocity and the temperature are kept, that of the
 *                     pressure reversed (through the chain rule back to the
 *                     conservative derivatives).
 *   GKS_BC_MOVING_WALL non-slip adiabatic wall moving along itself with
 *                     params.wall_velocity U_w (the paper's driven lid; it
 *                     prints no ghost for it): the ghost has the interior
 *                     density and pressure and the velocity 2 U_w - U; the
 *                     velocity derivatives are kept, those of density and
 *                     pressure reversed.  At U_w = 0 it is GKS_BC_NOSLIP_WALL.
 * The interior reconstruction of a boundary cell is the one-sided one of
 * Sec. 4.4 without constraint rows (for the non-slip wall the paper adds the
 * wall velocity as a constraint; this library does not): the cell's stencil
 * simply lacks the missing neighbour. */
enum { GKS_BC_OPEN = 0, GKS_BC_SLIP_WALL = 1, GKS_BC_FIXED = 2, GKS_BC_NOSLIP_WALL = 3,
       GKS_BC_ISOTHERMAL_WALL = 4, GKS_BC_MOVING_WALL = 5 };

/* kind[n_cell][4] (host): the condition of local face f (the face opposite
 * tet vertex f) of each cell, read only where that face is a boundary face.
 * Applies to states created afterwards (and to gks_workspace_bytes).  GKS_E_ARG on a NULL argument or an
 * unknown kind on a boundary face (the mesh keeps its previous kinds). */
gks_status gks_mesh_set_boundary(gks_mesh* mesh, const int8_t* kind);

/* Number of cases and case_first_cell[n_case + 1] (first cell of each case
 * and n_cell at the end; may be NULL). */
gks_status gks_mesh_cases(const gks_mesh* mesh, int32_t* n_case, int64_t* case_first_cell);

/* Counts: cells, faces, open boundary faces. Any output may be NULL. */
gks_status gks_mesh_info(const gks_mesh* mesh, int64_t* n_cell, int64_t* n_face,
                         int64_t* n_boundary_face);

/* Host copies of the connectivity (any output may be NULL):
 *   face_v[nf][3] ascending vertex ids; face_lr[nf][2] left and right cell
 *   (-1: none); nbr[nc][4] cell across the face opposite local vertex f
 *   (-1: none); csr_face[nc][4] face ids in local-face order; csr_sign[nc][4]
 *   +1 if the cell is that face's left cell, else -1. */
gks_status gks_mesh_topology(const gks_mesh* mesh, int64_t* face_v, int64_t* face_lr,
                             int64_t* nbr, int64_t* csr_face, int8_t* csr_sign);

/* Host copies of the FP64 geometry (any output may be NULL):
 *   vol[nc]; cen[nc][3]; mom2[nc][6] central second moments / volume in the
 *   order xx, xy, xz, yy, yz, zz; dr[nc] = 3|Omega| / sum |Gamma| (Sec. 5);
 *   farea[nf]; fnorm[nf][3]; gp_l[nf][3][3] and gp_r[nf][3][3] the face's
 *   Gauss points (Sec. 2.1: (1/6,1/6), (2/3,1/6), (1/6,2/3), weight area/3)
 *   relative to the left / right centroid, periodic image applied. */
gks_status gks_mesh_geometry(const gks_mesh* mesh, double* vol, double* cen, double* mom2,
                             double* dr, double* farea, double* fnorm, double* gp_l,
                             double* gp_r);

/* FP64 least-squares operators of every cell (Sec. 4.1, Sec. 4.3):
 *   M1 (3x4): slopes of P1 from the neighbours' averages minus the own,
 *   least squares (Eq. p1-stenci-condition);
 *   M2 (9x16): the 9 coefficients of P2 in the zero-mean basis of Eq. base
 *   from [dQ_f (4); grad Q_{f,l} at 4 + 3 f + l (12)], neighbour averages
 *   exact and neighbour gradients in the least-squares sense
 *   (Eqs. large-stenci-condition-1/2).
 * Columns of absent neighbours are zero.  *n_singular (may be NULL) counts
 * cells whose system is singular (fewer than 3 neighbours or reciprocal
 * pivot ratio below 1e-12); such cells reconstruct a constant.  Returns
 * GKS_OK even when n_singular > 0. */
gks_status gks_stencil_build(gks_mesh* mesh, int64_t* n_singular);

/* Host copies of M1[nc][3][4] and M2[nc][9][16] (GKS_E_STENCIL if not built). */
gks_status gks_mesh_stencils(const gks_mesh* mesh, double* M1, double* M2);

/* The constrained operators of Sec. 4.4 that params.wall_constraint = 1
 * applies to the momenta of cells with non-slip adiabatic wall faces
 * (GKS_BC_NOSLIP_WALL, as set by gks_mesh_set_boundary), built from the
 * mesh's FP64 geometry on each call:
 *   W1[nc][3][5]:  step-1 slopes b = W1 [dQ_f (4); Q0], the least-squares
 *                  P1 that vanishes at each wall face's centroid;
 *   W2[nc][9][17]: step-2 coefficients a = W2 [dQ_f (4); grad Q_{f,l} (12);
 *                  Q0] in the zero-mean basis of M2, the P2 with the
 *                  neighbour averages exact, the neighbour gradients in the
 *                  least-squares sense and zero at each wall face's three
 *                  Gauss points;
 *   built[nc]:     1 where both were built; zero rows elsewhere (no wall
 *                  face, fewer than 3 neighbours + wall faces, more than 9
 *                  equality rows, or a singular system: such a cell keeps
 *                  its one-sided stencil).
 * Any output may be NULL; *n_built (may be NULL) receives the count. */
gks_status gks_mesh_wall_stencils(const gks_mesh* mesh, double* W1, double* W2, int8_t* built,
                                  int64_t* n_built);

/* --------------------------------------------------------------- state -- */

/* Bytes of device workspace needed for this mesh and parameter set
 * (0 on error). */
size_t gks_workspace_bytes(const gks_mesh* mesh, const gks_params* params);

/* Binds a state to a mesh (stencils must be built), a parameter set, a
 * device workspace (256-byte aligned, at least gks_workspace_bytes) and a
 * CUDA stream (cudaStream_t passed as void*; NULL = legacy default stream).
 * Uploads the mesh data into the workspace (synchronously).  The mesh must
 * outlive the state. */
gks_status gks_state_create(const gks_mesh* mesh, const gks_params* params,
                            void* d_workspace, size_t workspace_bytes, void* stream,
                            gks_state** out);
void gks_state_destroy(gks_state* state);

/* Sets the state that fixed boundary faces (GKS_BC_FIXED) hold, from device
 * arrays W[5][nc], dW[15][nc] (FP64; read at the interior cell of each fixed
 * face), independently of the evolving state: later gks_init_state and
 * gks_step_host calls no longer overwrite it.  A run of steps that each
 * re-initialise the state (gradients over chained steps) then sees the same
 * boundary as one long run.  GKS_E_ARG on NULL or on a mesh without fixed
 * faces.  Synchronises. */
gks_status gks_set_fixed_state(gks_state* state, const double* d_W, const double* d_dW);

/* Sets the cell averages and gradients from device arrays W[5][nc],
 * dW[15][nc] (FP64) and the time to 0. */
gks_status gks_init_state(gks_state* state, const double* d_W, const double* d_dW);

/* Advances nsteps two-stage steps (Sec. 3).  dt_fixed > 0 fixes the step;
 * otherwise each step takes the time-step rule of Sec. 5 from the current
 * averages (a device-side reduction, per case for a batch).  t_end > 0 clips
 * each case's step so that its time does not pass t_end (steps of a case
 * at t = t_end are no-ops).  The step
 * sequence is captured once into a CUDA graph per option set and replayed.
 * Returns after enqueueing; host outputs need gks_sync or gks_get_time. */
gks_status gks_step(gks_state* state, int32_t nsteps, double dt_fixed, double t_end);

/* Waits for the state's stream and reports deferred errors. */
gks_status gks_sync(gks_state* state);

/* Copies the current W, dW (FP64) to device arrays (either may be NULL). */
gks_status gks_get_state(const gks_state* state, double* d_W, double* d_dW);

/* Time and last step size of case 0 (host values; synchronises). */
gks_status gks_get_time(gks_state* state, double* t, double* dt_last);

/* Time and last step of every case, t[n_case] and dt_last[n_case] (host
 * arrays, either may be NULL; synchronises). */
gks_status gks_case_times(gks_state* state, double* t, double* dt_last);

/* The same step through host buffers: copies h_W[5][nc], h_dW[15][nc] from
 * host memory (pinned for asynchronous copies), sets the time to 0 as
 * gks_init_state does, advances nsteps, and copies the result to h_W_out,
 * h_dW_out; synchronises.  In-place is allowed. */
gks_status gks_step_host(gks_state* state, const double* h_W, const double* h_dW,
                         int32_t nsteps, double dt_fixed, double* h_W_out,
                         double* h_dW_out);

/* Kernel classes timed by gks_step_timed. */
enum {
    GKS_K_DT = 0,      /* time-step minimum and control update */
    GKS_K_SLOPES = 1,  /* reconstruction step 1, both stages */
    GKS_K_RECON = 2,   /* reconstruction step 2, both stages */
    GKS_K_FLUX1 = 3,   /* face flux, stage 1 */
    GKS_K_UPDATE1 = 4, /* cell update, stage 1 */
    GKS_K_FLUX2 = 5,   /* face flux, stage 2 */
    GKS_K_UPDATE2 = 6, /* cell update, stage 2 */
    GKS_K_STAGE1 = 7,  /* stage 1 as one launch (gks_state_set_fused) */
    GKS_K_STAGE2 = 8,  /* stage 2 as one launch */
    GKS_NKERNELS = 9
};

/* The same steps as gks_step, launched kernel by kernel (no graph) with a
 * CUDA event between consecutive launches on the state's stream; adds each
 * kernel class's device time in milliseconds to kernel_ms[GKS_NKERNELS]
 * and its launch count to launches[GKS_NKERNELS] (may be NULL).
 * Synchronises.  For profiling breakdowns; numerically identical to
 * gks_step. */
gks_status gks_step_timed(gks_state* state, int32_t nsteps, double dt_fixed, double t_end,
                          double* kernel_ms, int64_t* launches);

/* Time step of the Sec. 5 rule for the current averages (host value). */
gks_status gks_timestep(gks_state* state, double* dt);

/* Largest number of cells gks_timestep_noalloc accepts, in blocks of 256. */
#define GKS_NOALLOC_MAX_BLOCKS 8192

/* The time step of gks_timestep without a gks_state and without any device
 * allocation, for callers that are not allowed to allocate device memory
 * (for example while a CUDA stream is being captured, or when another
 * framework owns the device memory).  The paper has no counterpart: this is
 * an interface convenience.
 *   p       scheme parameters (gamma, cfl, mu, viscous are used)
 *   d_W     device FP64 cell averages W[5][n_cell]
 *   d_dr    device FP64 radii dr[n_cell] (gks_mesh_geometry's dr)
 *   d_dt    device FP64 scalar receiving C_CFL * min over cells
 *   stream  CUDA stream (cudaStream_t as void*; NULL = legacy default)
 * Enqueues two small kernels and returns without synchronising.  Its
 * scratch is a fixed device array of GKS_NOALLOC_MAX_BLOCKS doubles held by
 * every GPU that loads the library; n_cell above 256 * that count is
 * rejected with GKS_E_ARG, as is a current device ordinal of 64 or more
 * (the per-device address cache has 64 slots).  The first call on a
 * device resolves the array's address (cudaGetSymbolAddress) with that
 * device current, so make it before any stream capture.  The address is
 * cached per device for the life of the process and belongs to the device's
 * primary context: after cudaDeviceReset (or any other teardown of that
 * context) the cached address is stale, so do not call this function on a
 * device that was reset after its first call.  All calls share the array:
 * calls that overlap on the GPU (unordered streams) race.  Allocates
 * nothing, frees nothing. */
gks_status gks_timestep_noalloc(const gks_params* p, const double* d_W, const double* d_dr,
                                int64_t n_cell, double* d_dt, void* stream);

/* Per-component root mean square over cells of (W(t) - W_prev) / dt_last,
 * where W_prev is the state before the last step (host out_l2[5];
 * synchronises). */
gks_status gks_residual(gks_state* state, double* out_l2);

/* -------------------------------------------------------------- adjoint -- */

/* The paper differentiates nothing: this is the reverse (adjoint) mode of one
 * step, for gradients of an output of a run with respect to its initial
 * state.  Given the adjoint of the step's result, (lamW [5][nc], lamdW
 * [15][nc]) = d J / d (W^{n+1}, grad W^{n+1}), it returns d J / d (W^n,
 * grad W^n) in (lamW_out, lamdW_out), with the time step frozen at dt: the
 * transpose of the step's Jacobian at (d_W, d_dW) applied to (lamW, lamdW).
 * It first recomputes the step's two reconstructions from (d_W, d_dW), so a
 * run of N steps back-propagates from the N saved (or recomputed) states.
 * Supported: FP64 states (precision 0) with the third- or second-order
 * reconstruction with linear or WENO weights (the weights are differentiated,
 * |x|' taken as sign x), full or smooth flux, Euler or viscous, single-case
 * meshes, periodic or with open, slip-wall, non-slip (adiabatic or
 * isothermal) wall or fixed-state boundary faces (the last only with a fixed state set by
 * gks_set_fixed_state: it is then a constant of the step), any Prandtl
 * number; GKS_E_UNSUPPORTED otherwise.  A cell that
 * falls back to its average (the positivity check of Sec. 4.3) passes the
 * adjoint of its constant to its own average only; the fallback decision is
 * held fixed (piecewise derivative).  All arrays are
 * device FP64; d_scratch (gks_adjoint_workspace_bytes) is caller-allocated
 * device memory.  On return the state is initialised at (d_W, d_dW) with its
 * time reset.  Synchronises. */
size_t gks_adjoint_workspace_bytes(const gks_state* state);
gks_status gks_adjoint_step(gks_state* state, double dt, const double* d_W, const double* d_dW,
                            const double* d_lamW, const double* d_lamdW, double* d_lamW_out,
                            double* d_lamdW_out, void* d_scratch, size_t scratch_bytes);

/* The stage state of the last step of an FP64 state (precision 0): W*
 * [5][nc] and grad W* [15][nc] of the first stage of Eq. s2o4 as that step
 * computed them (device FP64, the caller's cell order).  GKS_E_UNSUPPORTED on
 * an FP32-bulk state, GKS_E_STATE when no step has run since the last
 * initialisation. */
gks_status gks_get_stage_state(gks_state* state, double* d_Ws, double* d_dWs);

/* gks_adjoint_step given the step's stage state (d_Ws, d_dWs), as
 * gks_get_stage_state returned it after the step from (d_W, d_dW) with the
 * same dt on a state of the same mesh and parameters: the forward
 * recomputation then skips the stage-1 flux and update and takes W*, grad W*
 * from the caller; everything else, and the result, is that of
 * gks_adjoint_step.  Same arguments and errors otherwise. */
gks_status gks_adjoint_step_staged(gks_state* state, double dt, const double* d_W, const double* d_dW,
                                   const double* d_Ws, const double* d_dWs, const double* d_lamW,
                                   const double* d_lamdW, double* d_lamW_out, double* d_lamdW_out,
                                   void* d_scratch, size_t scratch_bytes);

/* ---------------------------------------------------- tuning variants -- */

/* Execution variant of a state (the same arithmetic, only speed differs):
 *   face_order   0 = faces in canonical order, 1 = grouped by left cell
 *   flux_blocks  resident flux blocks per SM, 3 (more warps, fewer registers)
 *                or 2 (no register spills); FP32 only, ignored in FP64
 *   slopes_pass  0 = reconstruction step 1 (the P1 slopes, Sec. 4.3) is
 *                recomputed inside step 2 for each neighbour, 1 = a separate
 *                pass stores every cell's slopes first (WENO only)
 * Returns GKS_E_ARG for any other value.  Re-uploads the face arrays when the
 * order changes; the next gks_step captures a new graph. */
gks_status gks_state_set_variant(gks_state* state, int32_t face_order, int32_t flux_blocks,
                                 int32_t slopes_pass);

/* One launch per stage (precision 1 only): the reconstruction, the face
 * flux and the cell update of a stage run as one persistent kernel, one
 * block of 384 threads per SM striding over the blocks of cells and faces,
 * the three phases separated by grid-wide barriers (a cooperative launch,
 * so that every block is resident).  The same per-cell and per-face source
 * as the separate kernels; the compiler may contract or reorder a few FP32
 * operations differently in the one kernel, so results agree with the
 * separate kernels to FP32 rounding (not to the bit); flux_blocks and
 * slopes_pass do not apply.  Each barrier wait is
 * bounded: one that gives up makes the next synchronisation return
 * GKS_E_TIMEOUT.  GKS_E_ARG for another value, or for 1 on a state of
 * another precision.  The next gks_step captures a new graph. */
gks_status gks_state_set_fused(gks_state* state, int32_t fused);
gks_status gks_state_get_fused(const gks_state* state, int32_t* fused);

/* Number of execution variants gks_autotune times (entries of ms_per_step). */
enum { GKS_NVARIANTS = 10 };

/* Times every variant for `steps` steps on this state's own mesh and data,
 * keeps the fastest, and restores the state (averages, gradients, case times)
 * to what it was before the call.  Outputs (may be NULL): the chosen
 * face_order, flux_blocks and slopes_pass (the fused choice is read back by
 * gks_state_get_fused), and ms_per_step[GKS_NVARIANTS]: for v < 8 variant
 * v = face_order + 2 slopes_pass + 4 (3 - flux_blocks) with separate
 * kernels (the first 4 entries only in FP64, whose flux has one form); for
 * v = 8, 9 one launch per stage with face_order v - 8 (precision 1 only);
 * NaN for variants not timed.  Synchronises. */
gks_status gks_autotune(gks_state* state, int32_t steps, int32_t* face_order, int32_t* flux_blocks,
                        int32_t* slopes_pass, double* ms_per_step);

/* Cell ordering of the state's device arrays (FP32-bulk states, precision 1
 * or 2): 0 the caller's order, 1 reverse Cuthill-McKee on the face-neighbour
 * graph, 2 Morton (Z) order of the centroids; either taken within each case,
 * the cases staying contiguous.  An implementation choice for memory
 * locality that the paper does not discuss; every interface still speaks the
 * caller's cell order (states, gradients, diagnostics), and results are
 * bit-identical across orderings (every cell and face computes the same
 * arithmetic in the same order).  Changing the order of an initialised state
 * carries its averages, working state and fixed state over exactly;
 * synchronises.  GKS_E_ARG for another order, GKS_E_UNSUPPORTED for a
 * non-zero order on an FP64 state.  The next gks_step captures a new graph. */
gks_status gks_state_set_cell_order(gks_state* state, int32_t order);
gks_status gks_state_get_cell_order(const gks_state* state, int32_t* order);

/* gks_autotune over the cell orderings as well: for each ordering (FP64:
 * the caller's only) times every variant, keeps the fastest ordering and
 * variant (the fused choice included), and restores the state.  Outputs
 * (may be NULL): the chosen cell_order, face_order, flux_blocks, slopes_pass,
 * and ms_per_order[3], the best step time of each ordering.  Synchronises. */
gks_status gks_autotune_orders(gks_state* state, int32_t steps, int32_t* cell_order, int32_t* face_order,
                               int32_t* flux_blocks, int32_t* slopes_pass, double* ms_per_order);

/* ------------------------------------------------------- diagnostics -- */

/* Reconstruction of the current state (Sec. 4), written to device arrays:
 * d_poly[nc][5][10] R about each centroid in monomial form
 * (c0, cx, cy, cz, cxx, cxy, cxz, cyy, cyz, czz); d_slopes[nc][5][3] step-1
 * slopes (may be NULL; zero with linear weights); d_fallback[nc] 1 where the
 * positivity check replaced R by the average (may be NULL).  FP64 outputs
 * in both precisions. */
gks_status gks_debug_reconstruct(gks_state* state, double* d_poly, double* d_slopes,
                                 int32_t* d_fallback);

/* Face records of one stage for the current state and a given dt, written as
 * FP64 to d_rec[nf][40] (stage 1) or d_rec[nf][20] (stage 2), same layout as
 * used by the step: stage 1 = (sum_k w Fh, sum_k w (8/3 Fh - 1/3 F),
 * sum_k w (W0+Wdt)/2 n, sum_k w W0 n); stage 2 = (sum_k w 4/3 (F - 2 Fh),
 * sum_k w (Wdt - W0) n); vector entries at 3*q + i.  Fh, F are the flux
 * integrals over [0, dt/2] and [0, dt]; W0, Wdt the interface states
 * (Sec. 2.2, Sec. 3 Eqs. linear-system, step-du). */
gks_status gks_debug_face_records(gks_state* state, double dt, int32_t stage, double* d_rec);

/* Failure path of the bounded device waits, without a fault: runs the
 * reconstruction's mbarrier wait on a barrier that no copy completes
 * (nothing is in flight), polling it `tries` times (0..65536); the give-up
 * sets the state's device error flag as a stalled tile copy would.  Returns
 * what the next synchronisation reports (GKS_E_TIMEOUT), then clears the
 * flag so that the state stays usable.  Synchronises.  For tests. */
gks_status gks_debug_wait_timeout(gks_state* state, int32_t tries);

/* The same for the one-launch stage's grid-wide barrier (gks_state_set_fused):
 * two blocks wait on a barrier that no arrival can complete, each polling
 * `tries` times (0..65536) before it gives up and sets the error flag, as a
 * stage whose blocks were not all resident would.  Returns what the next
 * synchronisation reports (GKS_E_TIMEOUT), then clears the flag.  Any
 * precision.  Synchronises.  For tests. */
gks_status gks_debug_grid_barrier_timeout(gks_state* state, int32_t tries);

/* Last error message of this thread ("" if none). */
const char* gks_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GKS_H */
