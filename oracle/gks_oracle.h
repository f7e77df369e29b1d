/*
 * gks_oracle.h -- plain FP64 CPU oracle of the two-stage compact gas-kinetic
 * scheme with two-step multi-resolution WENO reconstruction on tetrahedra.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this code.  It shares no code with
 * the CUDA library; the two meet only in the seeded input generator.
 *
 * Every array is row-major FP64 unless stated; "nc" cells, "nf" faces.
 * State layout: W[5][nc] conservative (rho, rho U1, rho U2, rho U3, rho E);
 * dW[15][nc] with row 3*q+i = d W_q / d x_i (cell-averaged gradients).
 */
#ifndef GKS_ORACLE_H
#define GKS_ORACLE_H
#include <stdint.h>

typedef struct {
    double gamma;      /* specific heat ratio */
    double cfl;        /* C_CFL of the time-step rule, Sec. 5 */
    double mu;         /* dynamic viscosity (viscous only) */
    double eps_weno;   /* epsilon of the nonlinear weights, Sec. 4.2 (1e-8) */
    double tau_eps;    /* epsilon of the numerical collision time, Sec. 2.2 (0.01) */
    double tau_c;      /* C of the numerical collision time (1) */
    int32_t weno;      /* 0: linear weights (R = P2), 1: nonlinear weights */
    int32_t order;     /* 3: third-order R, 2: second-order R (Eq. of R^2nd) */
    int32_t smooth_flux; /* 0: full solver (2nd-flux), 1: smooth solver */
    int32_t viscous;   /* 0: Euler (tau = 0), 1: tau = mu / p */
    double prandtl;    /* viscous only: Pr != 1 corrects the heat flux (Pr fix) */
    double wall_temperature; /* T = p / rho of isothermal walls */
    double wall_velocity[3]; /* velocity of moving walls (global frame) */
    int32_t wall_constraint; /* 1: Sec. 4.4 constrained least squares for the
                                momenta of cells with non-slip adiabatic wall
                                faces (velocity zero at the wall); 0: the
                                unconstrained one-sided stencil */
} ora_params;

typedef struct ora_mesh ora_mesh;

/* Builds topology, geometry and stencil matrices.  shift[nc][4][3] are the
 * periodic image shifts of the tet vertices; period[a] == 0 on a
 * non-periodic axis.  Returns NULL and writes a message on error. */
ora_mesh* ora_mesh_build(const double* xyz, int64_t nv, const int64_t* tet,
                         const int8_t* shift, int64_t nc, const double* period,
                         char* err, int errlen);
void ora_mesh_free(ora_mesh* m);

/* Boundary condition of the boundary faces (faces with one cell). */
enum { ORA_BC_OPEN = 0, ORA_BC_SLIP_WALL = 1, ORA_BC_FIXED = 2, ORA_BC_NOSLIP_WALL = 3,
       ORA_BC_ISOTHERMAL_WALL = 4, ORA_BC_MOVING_WALL = 5 };
/* kind[nc][4]: the condition of local face f (opposite vertex f) of cell c,
 * read only where that face is on the boundary.  Default: all open.
 * Returns -1 (mesh unchanged only up to the offending face) on a value
 * that is not one of ORA_BC_*. */
int ora_mesh_set_boundary(ora_mesh* m, const int8_t* kind);
/* The state a fixed boundary (ORA_BC_FIXED) holds: W[5][nc], dW[15][nc] of
 * the cells (read at the interior cell of each fixed face; copied).  Face
 * records and steps return -1 while a fixed face has no state. */
void ora_mesh_set_fixed_state(ora_mesh* m, const double* W, const double* dW);
int64_t ora_mesh_nc(const ora_mesh* m);
int64_t ora_mesh_nf(const ora_mesh* m);
int64_t ora_mesh_n_singular(const ora_mesh* m);

/* face_v[nf][3] sorted vertex ids; face_lr[nf][2] (left, right; -1 = none);
 * nbr[nc][4] cell across the face opposite local vertex f (-1 = none);
 * csr_face[nc][4] face ids in local-face order; csr_sign[nc][4] +1 if the
 * cell is the face's left cell, else -1. */
void ora_mesh_topology(const ora_mesh* m, int64_t* face_v, int64_t* face_lr,
                       int64_t* nbr, int64_t* csr_face, int8_t* csr_sign);
/* vol[nc], cen[nc][3], mom2[nc][6] (xx,xy,xz,yy,yz,zz central second
 * moments / vol), dr[nc]; farea[nf], fnorm[nf][3] (left -> right),
 * gp_l[nf][3][3], gp_r[nf][3][3] Gauss points relative to the left / right
 * centroid (periodic image applied); rows of absent cells are zero. */
void ora_mesh_geometry(const ora_mesh* m, double* vol, double* cen, double* mom2,
                       double* dr, double* farea, double* fnorm, double* gp_l,
                       double* gp_r);
/* M1[nc][3][4], M2[nc][9][16]; columns of absent neighbours are zero. */
void ora_mesh_stencils(const ora_mesh* m, double* M1, double* M2);

/* The constrained stencils of Sec. 4.4 at non-slip adiabatic walls (built
 * by ora_mesh_set_boundary for every cell with an ORA_BC_NOSLIP_WALL face):
 * MW1[nc][3][5] gives a momentum component's step-1 slopes as
 * b = MW1 [dQ_f (4); Q0], the P1 of the least-squares fit to the
 * neighbours' averages that vanishes at the centroid of each wall face;
 * MW2[nc][9][17] gives its P2 coefficients (zero-mean basis, as M2) as
 * a = MW2 [data (16); Q0], P2 fitted like the unconstrained one and
 * vanishing at the three Gauss points of each wall face.  wallc[nc] is 1
 * where both were built, else 0 (no wall face, too few data, or a singular
 * system: the cell keeps its unconstrained stencils).  Any output may be
 * NULL.  Returns the number of cells with wallc = 1. */
int64_t ora_mesh_wall_stencils(const ora_mesh* m, double* MW1, double* MW2, int8_t* wallc);

/* Reconstruction of every cell.  poly[nc][5][10] is R in centroid-monomial
 * form: c0 + c_x X + c_y Y + c_z Z + c_xx X^2 + c_xy XY + c_xz XZ + c_yy Y^2
 * + c_yz YZ + c_zz Z^2 with X = x - centroid.  slopes[nc][5][3] (may be
 * NULL) are the step-1 slopes.  fallback[nc] (may be NULL) is 1 where the
 * positivity check replaced R by the cell average. */
int ora_reconstruct(const ora_mesh* m, const ora_params* p, const double* W,
                    const double* dW, double* poly, double* slopes,
                    int32_t* fallback);

/* Pieces of the reconstruction, exposed so that tests can pin them:
 * ora_smoothness: the smoothness indicator of Eq. smooth-indicator (Sec. 4.2)
 * of cell c for a polynomial v[10] in the cell's zero-mean basis form
 * (v[0] constant, v[1..3] linear, v[4..9] the quadratic basis in the order
 * xx, xy, xz, yy, yz, zz), r = 1 (first derivatives only) or 2.
 * ora_weno_beta0: beta_0 of Sec. 4.3 (Eq. p0-non-linear-weight) from the
 * step-1 slopes b[nn][3] of nn <= 4 neighbours on a cell of volume vol;
 * sigma1 and wbar1[nn] (may be NULL) receive sigma^1st and the normalised
 * weights omega-bar^1st_j.
 * ora_weno_weights: the normalised nonlinear weights (Eq. non-linear-weight)
 * of p_0, p_1 (order 2) or p_0, p_1, p_2 (order 3) into wbar[3]. */
double ora_smoothness(const ora_mesh* m, int64_t c, const double* v, int r);
double ora_weno_beta0(double vol, const double* b, int nn, double eps, double* sigma1, double* wbar1);
void ora_weno_weights(int order, double eps, double beta0, double beta1, double beta2, double* wbar);

/* Time-dependent kinetic solution at one Gauss point, everything in the local
 * face frame (x1 along the normal).  dWl[i][q] = d W_q / d x_i.  Outputs the
 * time integrals of the flux over [0, dt/2] and [0, dt] and the point values
 * W(0), W(dt); each 5 long. */
void ora_gp_flux(const ora_params* p, const double* Wl, const double* dWl,
                 const double* Wr, const double* dWr, double dt,
                 double* Fh, double* F, double* W0, double* Wdt);

/* Face records of one stage.  Stage 1: rec[nf][40] = (sum w Fh (5),
 * sum w (8/3 Fh - 1/3 F) (5), sum w (W0+Wdt)/2 n (15), sum w W0 n (15)).
 * Stage 2: rec[nf][20] = (sum w 4/3 (F - 2 Fh) (5), sum w (Wdt - W0) n (15)).
 * Vector-valued entries are stored component-major: 3*q + i. */
int ora_face_records(const ora_mesh* m, const ora_params* p, const double* W,
                     const double* dW, double dt, int stage, double* rec);

/* Global time step (Sec. 5 time-step rule) from the cell averages. */
double ora_timestep(const ora_mesh* m, const ora_params* p, const double* W);

/* One two-stage step in place.  dt <= 0: use the time-step rule.  Returns
 * the step used in *dt_used.  Returns 0 on success. */
int ora_step(const ora_mesh* m, const ora_params* p, double* W, double* dW,
             double dt, double* dt_used);

/* The stage-assembly helpers of ora_step applied to the scalar linear ODE
 * y' = z y / dt, each stage's flux linear in time with its exact
 * instantaneous derivative; returns y(dt) / y(0). */
double ora_s2o4_linear_ode(double z);

#endif
