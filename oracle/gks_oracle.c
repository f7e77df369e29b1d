/*
 * gks_oracle.c -- plain FP64 CPU oracle of one two-stage step of the
 * third-order compact gas-kinetic scheme on tetrahedral meshes (Ji, Zhao,
 * Shyy, Xu, "Two-step multi-resolution reconstruction-based compact
 * gas-kinetic scheme on tetrahedral mesh").
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
 * CPU-baseline leg are the only users.  It is written for clarity, not speed:
 * velocity-space moments are evaluated term by term from sparse polynomials,
 * micro-slopes come from a direct 5x5 linear solve, least-squares stencils
 * from a dense KKT solve, smoothness indicators from a volume quadrature.
 *
 * Section / equation map:
 *   mesh, faces, Gauss points ......... Sec. 2.1 (face rule, Eq. fv-3d-general)
 *   cell moments (5-point rule) ....... Sec. 4.1 (Eq. base-int-change)
 *   local frame T ..................... Sec. 2.1 (Eq. rotate-3d, rotate-matrix-3d)
 *   micro-slopes, A ................... Sec. 2.2 (Eq. co)
 *   equilibrium state g^c ............. Sec. 4.5 (Eq. new-equ-part)
 *   time-dependent f .................. Sec. 2.2 (Eq. 2nd-flux, 2nd-smooth-flux)
 *   collision times ................... Sec. 2.2 (tau_n rule)
 *   interface gradient update ......... Sec. 2.3 (Eq. gauss-formula) and Sec. 3
 *                                        (Eq. step-du)
 *   S2O4 stages, linear flux fit ....... Sec. 3 (Eq. s2o4, linear-system)
 *   P2 / P1 / P0 stencils ............. Sec. 4.1 (Eqs. large-stenci-condition,
 *                                        p1-stenci-condition)
 *   multi-resolution WENO ............. Sec. 4.2 (Eqs. smooth-indicator,
 *                                        non-linear-weight, final_weno_expression)
 *   two-step beta_0 ................... Sec. 4.3 (Eq. p0-non-linear-weight)
 *   time step ......................... Sec. 5 (Eq. time-step)
 *
 * Readings where the paper is silent or garbled are listed in the design
 * notes; each is marked READING below.
 */
#include "gks_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORA_PI 3.14159265358979323846

struct ora_mesh {
    int64_t nv, nc, nf;
    double period[3];
    double* xyz;
    int64_t* tet;
    int8_t* shift;
    /* topology */
    int64_t* face_v;    /* [nf][3] */
    int64_t* face_lr;   /* [nf][2] */
    int64_t* nbr;       /* [nc][4] */
    int64_t* nbr_shift; /* [nc][4][3] image shift, cell frame -> neighbour */
    int64_t* csr_face;  /* [nc][4] */
    int8_t* csr_sign;   /* [nc][4] */
    /* geometry */
    double *vol, *cen, *mom2, *dr;
    double *farea, *fnorm, *gp_l, *gp_r;
    /* stencils */
    double *M1, *M2;
    double* M2L;  /* [nc][3][16]: boundary cells' first-order fit (Sec. 4.4), else 0 */
    int64_t n_singular;
    /* Sec. 4.4 constrained stencils of cells with non-slip adiabatic wall
     * faces (built with the boundary kinds) */
    double* MW1;     /* [nc][3][5] */
    double* MW2;     /* [nc][9][17] */
    int8_t* wallc;   /* [nc] 1 where built */
    /* boundary kind of each face (ORA_BC_*), meaningful on boundary faces */
    int8_t* bkind;      /* [nf] */
    /* the fixed boundary state: a copy of W[5][nc], dW[15][nc] (or NULL) */
    double *fixW, *fixdW;
};

/* ------------------------------------------------------------------------ */
/* small dense linear algebra                                               */
/* ------------------------------------------------------------------------ */

/* Gaussian elimination with partial pivoting: A (n x n) X = B (n x nrhs),
 * both row-major, overwritten; X returned in B.  Reports the smallest and
 * largest pivot magnitudes.  Returns -1 on an exactly zero pivot. */
static int gauss_solve(int n, int nrhs, double* A, double* B, double* pmin,
                       double* pmax) {
    double lo = INFINITY, hi = 0.0;
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int r = k + 1; r < n; ++r)
            if (fabs(A[r * n + k]) > fabs(A[p * n + k])) p = r;
        if (A[p * n + k] == 0.0) return -1;
        if (p != k) {
            for (int c = 0; c < n; ++c) {
                double t = A[k * n + c]; A[k * n + c] = A[p * n + c]; A[p * n + c] = t;
            }
            for (int c = 0; c < nrhs; ++c) {
                double t = B[k * nrhs + c]; B[k * nrhs + c] = B[p * nrhs + c]; B[p * nrhs + c] = t;
            }
        }
        double piv = A[k * n + k];
        if (fabs(piv) < lo) lo = fabs(piv);
        if (fabs(piv) > hi) hi = fabs(piv);
        for (int r = k + 1; r < n; ++r) {
            double f = A[r * n + k] / piv;
            if (f == 0.0) continue;
            for (int c = k; c < n; ++c) A[r * n + c] -= f * A[k * n + c];
            for (int c = 0; c < nrhs; ++c) B[r * nrhs + c] -= f * B[k * nrhs + c];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        for (int c = 0; c < nrhs; ++c) {
            double s = B[k * nrhs + c];
            for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * B[j * nrhs + c];
            B[k * nrhs + c] = s / A[k * n + k];
        }
    }
    if (pmin) *pmin = lo;
    if (pmax) *pmax = hi;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* mesh: topology                                                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t v[3];   /* face vertex ids, ascending */
    int rel[6];     /* image shift of v[1], v[2] relative to v[0] */
    int64_t cell;
    int local;      /* local face = local vertex opposite */
    int sa[3];      /* image shift of v[0] inside this cell */
} side_rec;

static int cmp_key(const side_rec* a, const side_rec* b) {
    for (int i = 0; i < 3; ++i)
        if (a->v[i] != b->v[i]) return a->v[i] < b->v[i] ? -1 : 1;
    for (int i = 0; i < 6; ++i)
        if (a->rel[i] != b->rel[i]) return a->rel[i] < b->rel[i] ? -1 : 1;
    return 0;
}

static int cmp_side(const void* pa, const void* pb) {
    const side_rec* a = (const side_rec*)pa;
    const side_rec* b = (const side_rec*)pb;
    int c = cmp_key(a, b);
    if (c) return c;
    if (a->cell != b->cell) return a->cell < b->cell ? -1 : 1;
    return a->local - b->local;
}

/* position of local vertex v of cell c in the cell's own frame */
static void cell_vertex(const ora_mesh* m, int64_t c, int v, double x[3]) {
    int64_t id = m->tet[c * 4 + v];
    for (int a = 0; a < 3; ++a)
        x[a] = m->xyz[id * 3 + a] + (double)m->shift[(c * 4 + v) * 3 + a] * m->period[a];
}

static void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* 3-point face rule, Sec. 2.1: (xi, eta) = (1/6,1/6), (2/3,1/6), (1/6,2/3),
 * weights 1/3 of the reference area. */
static const double GP_XI[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
static const double GP_ETA[3] = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};

/* 5-point volume rule, Sec. 4.1.  READING: the printed weights (-1/5 and
 * 3/40) do not sum to the reference volume 1/6; the degree-3 rule with these
 * points has -2/15 at the centre and 3/40 elsewhere. */
static const double VQ_P[5][3] = {{0.25, 0.25, 0.25},
                                  {0.5, 1.0 / 6.0, 1.0 / 6.0},
                                  {1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0},
                                  {1.0 / 6.0, 1.0 / 6.0, 0.5},
                                  {1.0 / 6.0, 0.5, 1.0 / 6.0}};
static const double VQ_W[5] = {-2.0 / 15.0, 3.0 / 40.0, 3.0 / 40.0, 3.0 / 40.0, 3.0 / 40.0};

static void set_err(char* err, int errlen, const char* msg) {
    if (err && errlen > 0) {
        strncpy(err, msg, (size_t)errlen - 1);
        err[errlen - 1] = 0;
    }
}

static int build_topology(ora_mesh* m, char* err, int errlen) {
    int64_t ns = m->nc * 4;
    side_rec* s = (side_rec*)calloc((size_t)ns, sizeof(side_rec));
    if (!s) { set_err(err, errlen, "out of memory"); return -1; }
    for (int64_t c = 0; c < m->nc; ++c) {
        for (int f = 0; f < 4; ++f) {
            int loc[3], k = 0;
            for (int v = 0; v < 4; ++v) if (v != f) loc[k++] = v;
            /* sort the three local vertices by global id */
            for (int i = 0; i < 3; ++i)
                for (int j = i + 1; j < 3; ++j)
                    if (m->tet[c * 4 + loc[j]] < m->tet[c * 4 + loc[i]]) {
                        int t = loc[i]; loc[i] = loc[j]; loc[j] = t;
                    }
            side_rec* r = &s[c * 4 + f];
            for (int i = 0; i < 3; ++i) r->v[i] = m->tet[c * 4 + loc[i]];
            if (r->v[0] == r->v[1] || r->v[1] == r->v[2]) {
                set_err(err, errlen, "tetrahedron repeats a vertex id");
                free(s);
                return -1;
            }
            for (int a = 0; a < 3; ++a) {
                int s0 = m->shift[(c * 4 + loc[0]) * 3 + a];
                r->sa[a] = s0;
                r->rel[a] = m->shift[(c * 4 + loc[1]) * 3 + a] - s0;
                r->rel[3 + a] = m->shift[(c * 4 + loc[2]) * 3 + a] - s0;
            }
            r->cell = c;
            r->local = f;
        }
    }
    qsort(s, (size_t)ns, sizeof(side_rec), cmp_side);
    int64_t nf = 0;
    for (int64_t i = 0; i < ns;) {
        int64_t j = i + 1;
        while (j < ns && cmp_key(&s[i], &s[j]) == 0) ++j;
        if (j - i > 2) {
            set_err(err, errlen, "face shared by more than two cells");
            free(s);
            return -1;
        }
        ++nf;
        i = j;
    }
    m->nf = nf;
    m->face_v = (int64_t*)malloc(sizeof(int64_t) * 3 * nf);
    m->face_lr = (int64_t*)malloc(sizeof(int64_t) * 2 * nf);
    m->bkind = (int8_t*)calloc((size_t)nf, sizeof(int8_t));
    m->farea = (double*)calloc((size_t)nf, sizeof(double));
    m->fnorm = (double*)calloc((size_t)nf * 3, sizeof(double));
    m->gp_l = (double*)calloc((size_t)nf * 9, sizeof(double));
    m->gp_r = (double*)calloc((size_t)nf * 9, sizeof(double));
    m->nbr = (int64_t*)malloc(sizeof(int64_t) * 4 * m->nc);
    m->nbr_shift = (int64_t*)calloc((size_t)m->nc * 12, sizeof(int64_t));
    m->csr_face = (int64_t*)malloc(sizeof(int64_t) * 4 * m->nc);
    m->csr_sign = (int8_t*)malloc(sizeof(int8_t) * 4 * m->nc);
    for (int64_t i = 0; i < 4 * m->nc; ++i) m->nbr[i] = -1;

    int64_t fi = 0;
    for (int64_t i = 0; i < ns; ++fi) {
        int64_t j = i + 1;
        while (j < ns && cmp_key(&s[i], &s[j]) == 0) ++j;
        const side_rec* r0 = &s[i];
        for (int k = 0; k < 3; ++k) m->face_v[fi * 3 + k] = r0->v[k];
        /* face frame: v0 at its base position, v1, v2 by relative shift */
        double xa[3], xb[3], xc[3], e1[3], e2[3], n[3];
        for (int a = 0; a < 3; ++a) {
            xa[a] = m->xyz[r0->v[0] * 3 + a];
            xb[a] = m->xyz[r0->v[1] * 3 + a] + (double)r0->rel[a] * m->period[a];
            xc[a] = m->xyz[r0->v[2] * 3 + a] + (double)r0->rel[3 + a] * m->period[a];
            e1[a] = xb[a] - xa[a];
            e2[a] = xc[a] - xa[a];
        }
        cross3(e1, e2, n);
        /* READING: canonical orientation, first nonzero component positive */
        int positive = n[0] > 0.0 || (n[0] == 0.0 && (n[1] > 0.0 || (n[1] == 0.0 && n[2] > 0.0)));
        if (!positive) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
        double nn = sqrt(dot3(n, n));
        if (!(nn > 0.0)) {
            set_err(err, errlen, "degenerate face");
            free(s);
            return -1;
        }
        m->farea[fi] = 0.5 * nn;
        for (int a = 0; a < 3; ++a) m->fnorm[fi * 3 + a] = n[a] / nn;
        m->face_lr[fi * 2] = -1;
        m->face_lr[fi * 2 + 1] = -1;
        int sa_side[2][3];
        int local_side[2] = {-1, -1};
        for (int q = 0; q < 3; ++q) { sa_side[0][q] = 0; sa_side[1][q] = 0; }
        for (int64_t t = i; t < j; ++t) {
            const side_rec* r = &s[t];
            int64_t c = r->cell;
            double xo[3], d[3];
            int64_t o = m->tet[c * 4 + r->local];
            for (int a = 0; a < 3; ++a) {
                xo[a] = m->xyz[o * 3 + a] +
                        (double)(m->shift[(c * 4 + r->local) * 3 + a] - r->sa[a]) * m->period[a];
                d[a] = xo[a] - xa[a];
            }
            double side = dot3(d, n);
            int lr;
            if (side < 0.0) lr = 0;       /* n points out of this cell: left */
            else if (side > 0.0) lr = 1;  /* right */
            else { set_err(err, errlen, "flat tetrahedron"); free(s); return -1; }
            if (m->face_lr[fi * 2 + lr] != -1) {
                set_err(err, errlen, "both cells on the same side of a face");
                free(s);
                return -1;
            }
            m->face_lr[fi * 2 + lr] = c;
            local_side[lr] = r->local;
            for (int a = 0; a < 3; ++a) sa_side[lr][a] = r->sa[a];
            m->csr_face[c * 4 + r->local] = fi;
            m->csr_sign[c * 4 + r->local] = (int8_t)(lr == 0 ? 1 : -1);
        }
        if (j - i == 2) {
            int64_t cl = m->face_lr[fi * 2], cr = m->face_lr[fi * 2 + 1];
            m->nbr[cl * 4 + local_side[0]] = cr;
            m->nbr[cr * 4 + local_side[1]] = cl;
            for (int a = 0; a < 3; ++a) {
                m->nbr_shift[(cl * 4 + local_side[0]) * 3 + a] = sa_side[0][a] - sa_side[1][a];
                m->nbr_shift[(cr * 4 + local_side[1]) * 3 + a] = sa_side[1][a] - sa_side[0][a];
            }
        }
        /* Gauss points in the face frame, then relative to each centroid
         * (filled after cell geometry is known; store the face-frame points
         * with the side shifts for now) */
        for (int k = 0; k < 3; ++k) {
            for (int a = 0; a < 3; ++a) {
                double x = xa[a] + GP_XI[k] * e1[a] + GP_ETA[k] * e2[a];
                m->gp_l[fi * 9 + k * 3 + a] = x + (double)sa_side[0][a] * m->period[a];
                m->gp_r[fi * 9 + k * 3 + a] = x + (double)sa_side[1][a] * m->period[a];
            }
        }
        i = j;
    }
    free(s);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* mesh: geometry                                                           */
/* ------------------------------------------------------------------------ */

static int build_geometry(ora_mesh* m, char* err, int errlen) {
    m->vol = (double*)malloc(sizeof(double) * m->nc);
    m->cen = (double*)malloc(sizeof(double) * 3 * m->nc);
    m->mom2 = (double*)malloc(sizeof(double) * 6 * m->nc);
    m->dr = (double*)malloc(sizeof(double) * m->nc);
    for (int64_t c = 0; c < m->nc; ++c) {
        double x[4][3];
        for (int v = 0; v < 4; ++v) cell_vertex(m, c, v, x[v]);
        double e1[3], e2[3], e3[3], cr[3];
        for (int a = 0; a < 3; ++a) {
            e1[a] = x[1][a] - x[0][a];
            e2[a] = x[2][a] - x[0][a];
            e3[a] = x[3][a] - x[0][a];
        }
        cross3(e2, e3, cr);
        double jac = dot3(e1, cr); /* = 6 |Omega| */
        if (!(jac > 0.0)) {
            set_err(err, errlen, "tetrahedron with non-positive volume");
            return -1;
        }
        double vol = jac / 6.0;
        m->vol[c] = vol;
        for (int a = 0; a < 3; ++a)
            m->cen[c * 3 + a] = 0.25 * (x[0][a] + x[1][a] + x[2][a] + x[3][a]);
        /* central second moments by the 5-point rule (exact for degree 2) */
        double M[6] = {0, 0, 0, 0, 0, 0};
        for (int q = 0; q < 5; ++q) {
            double y[3];
            for (int a = 0; a < 3; ++a)
                y[a] = x[0][a] + VQ_P[q][0] * e1[a] + VQ_P[q][1] * e2[a] + VQ_P[q][2] * e3[a] -
                       m->cen[c * 3 + a];
            double w = VQ_W[q] * jac / vol;
            M[0] += w * y[0] * y[0];
            M[1] += w * y[0] * y[1];
            M[2] += w * y[0] * y[2];
            M[3] += w * y[1] * y[1];
            M[4] += w * y[1] * y[2];
            M[5] += w * y[2] * y[2];
        }
        for (int k = 0; k < 6; ++k) m->mom2[c * 6 + k] = M[k];
    }
    /* Gauss points relative to centroids; inscribed-radius estimate */
    for (int64_t c = 0; c < m->nc; ++c) m->dr[c] = 0.0;
    for (int64_t f = 0; f < m->nf; ++f) {
        int64_t cl = m->face_lr[f * 2], cr = m->face_lr[f * 2 + 1];
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) {
                if (cl >= 0) m->gp_l[f * 9 + k * 3 + a] -= m->cen[cl * 3 + a];
                else m->gp_l[f * 9 + k * 3 + a] = 0.0;
                if (cr >= 0) m->gp_r[f * 9 + k * 3 + a] -= m->cen[cr * 3 + a];
                else m->gp_r[f * 9 + k * 3 + a] = 0.0;
            }
        if (cl >= 0) m->dr[cl] += m->farea[f];
        if (cr >= 0) m->dr[cr] += m->farea[f];
    }
    for (int64_t c = 0; c < m->nc; ++c) m->dr[c] = 3.0 * m->vol[c] / m->dr[c];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* mesh: stencil matrices, Sec. 4.1                                          */
/* ------------------------------------------------------------------------ */

/* quadratic basis pairs in the order xx, xy, xz, yy, yz, zz */
static const int QI[6] = {0, 0, 0, 1, 1, 2};
static const int QJ[6] = {0, 1, 2, 1, 2, 2};

static void neighbour_offset(const ora_mesh* m, int64_t c, int f, double d[3]) {
    int64_t nb = m->nbr[c * 4 + f];
    for (int a = 0; a < 3; ++a)
        d[a] = m->cen[nb * 3 + a] + (double)m->nbr_shift[(c * 4 + f) * 3 + a] * m->period[a] -
               m->cen[c * 3 + a];
}

static void build_stencils(ora_mesh* m) {
    m->M1 = (double*)calloc((size_t)m->nc * 12, sizeof(double));
    m->M2 = (double*)calloc((size_t)m->nc * 144, sizeof(double));
    m->M2L = (double*)calloc((size_t)m->nc * 48, sizeof(double));
    m->n_singular = 0;
    for (int64_t c = 0; c < m->nc; ++c) {
        int faces[4], nn = 0;
        double d[4][3];
        for (int f = 0; f < 4; ++f)
            if (m->nbr[c * 4 + f] >= 0) {
                faces[nn] = f;
                neighbour_offset(m, c, f, d[nn]);
                ++nn;
            }
        if (nn < 3) { ++m->n_singular; continue; }
        /* P1 (Eq. p1-stenci-condition): least squares on the neighbours'
         * averages, unweighted (READING).  M1 = (A^T A)^-1 A^T. */
        double N[9] = {0}, B[3 * 4] = {0};
        for (int r = 0; r < nn; ++r)
            for (int i = 0; i < 3; ++i) {
                for (int j = 0; j < 3; ++j) N[i * 3 + j] += d[r][i] * d[r][j];
                B[i * 4 + r] = d[r][i];
            }
        double pmin, pmax;
        if (gauss_solve(3, 4, N, B, &pmin, &pmax) != 0 || pmin < 1e-12 * pmax) {
            ++m->n_singular;
            continue;
        }
        for (int i = 0; i < 3; ++i)
            for (int r = 0; r < nn; ++r) m->M1[c * 12 + i * 4 + faces[r]] = B[i * 4 + r];

        /* P2 (Eqs. large-stenci-condition-1/2): neighbour averages exact,
         * neighbour averaged gradients in the least-squares sense (unweighted,
         * READING); the own cell average is built into the zero-mean basis.
         * Unknowns and rows are scaled by powers of h0 = |Omega|^(1/3) for
         * conditioning; the solution is unchanged. */
        double h0 = cbrt(m->vol[c]);
        double sc[9];
        for (int k = 0; k < 9; ++k) sc[k] = k < 3 ? h0 : h0 * h0;
        int n = 9 + nn;
        double K[13 * 13];
        double R[13 * 16];
        memset(K, 0, sizeof(K));
        memset(R, 0, sizeof(R));
        double Bm[12][9];
        const double* M0 = &m->mom2[c * 6];
        for (int r = 0; r < nn; ++r) {
            int64_t nb = m->nbr[c * 4 + faces[r]];
            const double* Mm = &m->mom2[nb * 6];
            double Crow[9];
            for (int k = 0; k < 3; ++k) Crow[k] = d[r][k] / sc[k];
            for (int q = 0; q < 6; ++q)
                Crow[3 + q] = (Mm[q] + d[r][QI[q]] * d[r][QJ[q]] - M0[q]) / sc[3 + q];
            for (int k = 0; k < 9; ++k) {
                K[(9 + r) * n + k] = Crow[k];
                K[k * n + 9 + r] = Crow[k];
            }
            for (int l = 0; l < 3; ++l) {
                double* row = Bm[r * 3 + l];
                for (int k = 0; k < 3; ++k) row[k] = h0 * (k == l ? 1.0 : 0.0) / sc[k];
                for (int q = 0; q < 6; ++q) {
                    double g = 0.0;
                    if (QI[q] == l) g += d[r][QJ[q]];
                    if (QJ[q] == l) g += d[r][QI[q]];
                    row[3 + q] = h0 * g / sc[3 + q];
                }
            }
        }
        int nrow = 3 * nn;
        for (int i = 0; i < 9; ++i)
            for (int j = 0; j < 9; ++j) {
                double s = 0.0;
                for (int r = 0; r < nrow; ++r) s += Bm[r][i] * Bm[r][j];
                K[i * n + j] = 2.0 * s;
            }
        /* right-hand sides: one column per data entry
         * (dQ_f for local face f; grad Q_{f,l} at 4 + 3 f + l) */
        for (int r = 0; r < nn; ++r) {
            R[(9 + r) * 16 + faces[r]] = 1.0;
            for (int l = 0; l < 3; ++l) {
                int col = 4 + 3 * faces[r] + l;
                for (int i = 0; i < 9; ++i) R[i * 16 + col] = 2.0 * Bm[r * 3 + l][i] * h0;
            }
        }
        if (gauss_solve(n, 16, K, R, &pmin, &pmax) != 0 || pmin < 1e-12 * pmax) {
            ++m->n_singular;
            memset(&m->M1[c * 12], 0, sizeof(double) * 12);
            continue;
        }
        for (int k = 0; k < 9; ++k)
            for (int j = 0; j < 16; ++j) m->M2[c * 144 + k * 16 + j] = R[k * 16 + j] / sc[k];

        /* Sec. 4.4: a boundary cell of the linear-weight (smooth)
         * reconstruction uses a first-order polynomial fitted to its P2
         * stencil in the least-squares sense.  READING: the rows are the
         * neighbours' averages (d_r . b = dQ_r) and averaged gradients
         * (b = grad Q_r, each scaled by h0 as in the P2 system), unweighted;
         * solved here by the normal equations. */
        if (nn == 3) {
            double G[9] = {0}, H[3 * 16] = {0};
            for (int r = 0; r < nn; ++r) {
                for (int i = 0; i < 3; ++i) {
                    for (int j = 0; j < 3; ++j) G[i * 3 + j] += d[r][i] * d[r][j] + (i == j ? h0 * h0 : 0.0);
                    H[i * 16 + faces[r]] = d[r][i];
                    H[i * 16 + 4 + 3 * faces[r] + i] = h0 * h0;
                }
            }
            if (gauss_solve(3, 16, G, H, &pmin, &pmax) == 0 && pmin >= 1e-12 * pmax)
                memcpy(&m->M2L[c * 48], H, sizeof(double) * 48);
        }
    }
}

/* Sec. 4.4, boundary cells at non-slip adiabatic walls: the momenta are
 * reconstructed by constrained least squares, the wall velocity (zero)
 * imposed on the polynomial at the wall faces, one point per face (its
 * centroid) in step 1 and the three Gauss points per face in step 2.  The
 * constraint value rho U_wall is zero whatever the density, so each
 * constrained polynomial is linear in the stencil data and the cell average
 * Q0: the operators below take Q0 as one more data column.
 *
 * Step 1: unknowns b (the slopes of P1(x) = Q0 + b.(x - x_c)); least-squares
 * rows d_r . b = dQ_r for the existing neighbours (as in the unconstrained
 * P1), equality rows e_w . b = -Q0 for each wall face w (e_w = its centroid
 * relative to the cell's).  Solved through the KKT system
 *   [sum d d^T  E^T] [b     ]   [sum d dQ]
 *   [E          0  ] [lambda] = [-Q0     ].
 * Used when neighbours + constraints >= 3 and constraints <= 3.
 *
 * Step 2: unknowns the nine zero-mean basis coefficients, as the
 * unconstrained P2: the neighbours' averages exact, their averaged gradients
 * in the least-squares sense, and P2(x_g) = 0 at each wall Gauss point
 * (sum_k a_k p^k(x_g) = -Q0) as further equality rows.  READING: the paper's
 * bullet for this case says "first-order polynomial"; its counts (data plus
 * constraints >= 9, constraints <= 9) are those of the nine P2 unknowns, and
 * its fallbacks are the first-order fits, so the constrained polynomial is
 * taken to be P2.  Built when the equality rows (neighbours + 3 x wall faces)
 * number at most 9 and neighbours + 3 x wall faces + 3 x neighbours >= 9.
 */
static void build_wall_stencils(ora_mesh* m) {
    free(m->MW1);
    free(m->MW2);
    free(m->wallc);
    m->MW1 = (double*)calloc((size_t)m->nc * 15, sizeof(double));
    m->MW2 = (double*)calloc((size_t)m->nc * 153, sizeof(double));
    m->wallc = (int8_t*)calloc((size_t)m->nc, 1);
    for (int64_t c = 0; c < m->nc; ++c) {
        int wf[4], nw = 0, faces[4], nn = 0;
        double d[4][3];
        for (int f = 0; f < 4; ++f) {
            if (m->nbr[c * 4 + f] >= 0) {
                faces[nn] = f;
                neighbour_offset(m, c, f, d[nn]);
                ++nn;
            } else if (m->bkind[m->csr_face[c * 4 + f]] == ORA_BC_NOSLIP_WALL) {
                wf[nw++] = f;
            }
        }
        if (nw == 0) continue;
        if (nn + nw < 3 || nw > 3 || nn + 3 * nw > 9 || nn + 3 * nw + 3 * nn < 9) continue;
        /* the wall faces' Gauss points relative to this cell's centroid */
        double xg[4][3][3], xc[4][3];
        for (int w = 0; w < nw; ++w) {
            int64_t fi = m->csr_face[c * 4 + wf[w]];
            const double* gp = m->csr_sign[c * 4 + wf[w]] > 0 ? &m->gp_l[fi * 9] : &m->gp_r[fi * 9];
            for (int a = 0; a < 3; ++a) {
                xc[w][a] = 0.0;
                for (int g = 0; g < 3; ++g) {
                    xg[w][g][a] = gp[g * 3 + a];
                    xc[w][a] += gp[g * 3 + a] / 3.0; /* the three points' mean is the centroid */
                }
            }
        }
        /* step 1 */
        int n1 = 3 + nw;
        double K1[6 * 6], R1[6 * 5], pmin, pmax;
        memset(K1, 0, sizeof(K1));
        memset(R1, 0, sizeof(R1));
        for (int r = 0; r < nn; ++r)
            for (int i = 0; i < 3; ++i) {
                for (int j = 0; j < 3; ++j) K1[i * n1 + j] += d[r][i] * d[r][j];
                R1[i * 5 + faces[r]] = d[r][i];
            }
        for (int w = 0; w < nw; ++w) {
            for (int i = 0; i < 3; ++i) {
                K1[(3 + w) * n1 + i] = xc[w][i];
                K1[i * n1 + 3 + w] = xc[w][i];
            }
            R1[(3 + w) * 5 + 4] = -1.0;
        }
        if (gauss_solve(n1, 5, K1, R1, &pmin, &pmax) != 0 || pmin < 1e-12 * pmax) continue;
        /* step 2 (unknowns and rows scaled by powers of h0 as in the
         * unconstrained P2; the solution is unchanged) */
        double h0 = cbrt(m->vol[c]);
        double sc[9];
        for (int k = 0; k < 9; ++k) sc[k] = k < 3 ? h0 : h0 * h0;
        int ne = nn + 3 * nw, n2 = 9 + ne;
        double K2[18 * 18], R2[18 * 17], Bm[12][9];
        memset(K2, 0, sizeof(K2));
        memset(R2, 0, sizeof(R2));
        const double* M0 = &m->mom2[c * 6];
        for (int r = 0; r < nn; ++r) {
            const double* Mm = &m->mom2[m->nbr[c * 4 + faces[r]] * 6];
            double row[9];
            for (int k = 0; k < 3; ++k) row[k] = d[r][k] / sc[k];
            for (int q = 0; q < 6; ++q) row[3 + q] = (Mm[q] + d[r][QI[q]] * d[r][QJ[q]] - M0[q]) / sc[3 + q];
            for (int k = 0; k < 9; ++k) {
                K2[(9 + r) * n2 + k] = row[k];
                K2[k * n2 + 9 + r] = row[k];
            }
            R2[(9 + r) * 17 + faces[r]] = 1.0;
            for (int l = 0; l < 3; ++l) {
                double* g = Bm[r * 3 + l];
                for (int k = 0; k < 3; ++k) g[k] = h0 * (k == l ? 1.0 : 0.0) / sc[k];
                for (int q = 0; q < 6; ++q) {
                    double v = 0.0;
                    if (QI[q] == l) v += d[r][QJ[q]];
                    if (QJ[q] == l) v += d[r][QI[q]];
                    g[3 + q] = h0 * v / sc[3 + q];
                }
            }
        }
        for (int w = 0; w < nw; ++w)
            for (int gpt = 0; gpt < 3; ++gpt) {
                const double* X = xg[w][gpt];
                int e = 9 + nn + 3 * w + gpt;
                double row[9];
                for (int k = 0; k < 3; ++k) row[k] = X[k] / sc[k];
                for (int q = 0; q < 6; ++q) row[3 + q] = (X[QI[q]] * X[QJ[q]] - M0[q]) / sc[3 + q];
                for (int k = 0; k < 9; ++k) {
                    K2[e * n2 + k] = row[k];
                    K2[k * n2 + e] = row[k];
                }
                R2[e * 17 + 16] = -1.0;
            }
        for (int i = 0; i < 9; ++i)
            for (int j = 0; j < 9; ++j) {
                double s = 0.0;
                for (int r = 0; r < 3 * nn; ++r) s += Bm[r][i] * Bm[r][j];
                K2[i * n2 + j] = 2.0 * s;
            }
        for (int r = 0; r < nn; ++r)
            for (int l = 0; l < 3; ++l)
                for (int i = 0; i < 9; ++i) R2[i * 17 + 4 + 3 * faces[r] + l] = 2.0 * Bm[r * 3 + l][i] * h0;
        if (gauss_solve(n2, 17, K2, R2, &pmin, &pmax) != 0 || pmin < 1e-12 * pmax) continue;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 5; ++j) m->MW1[c * 15 + i * 5 + j] = R1[i * 5 + j];
        for (int k = 0; k < 9; ++k)
            for (int j = 0; j < 17; ++j) m->MW2[c * 153 + k * 17 + j] = R2[k * 17 + j] / sc[k];
        m->wallc[c] = 1;
    }
}

int64_t ora_mesh_wall_stencils(const ora_mesh* m, double* MW1, double* MW2, int8_t* wallc) {
    int64_t n = 0;
    for (int64_t c = 0; c < m->nc; ++c) n += m->wallc && m->wallc[c];
    if (MW1) {
        if (m->MW1) memcpy(MW1, m->MW1, sizeof(double) * 15 * m->nc);
        else memset(MW1, 0, sizeof(double) * 15 * m->nc);
    }
    if (MW2) {
        if (m->MW2) memcpy(MW2, m->MW2, sizeof(double) * 153 * m->nc);
        else memset(MW2, 0, sizeof(double) * 153 * m->nc);
    }
    if (wallc) {
        if (m->wallc) memcpy(wallc, m->wallc, (size_t)m->nc);
        else memset(wallc, 0, (size_t)m->nc);
    }
    return n;
}

ora_mesh* ora_mesh_build(const double* xyz, int64_t nv, const int64_t* tet,
                         const int8_t* shift, int64_t nc, const double* period,
                         char* err, int errlen) {
    if (nc <= 0 || nc > ((int64_t)1 << 40) || nv <= 0) {
        set_err(err, errlen, "empty or oversized mesh");
        return NULL;
    }
    ora_mesh* m = (ora_mesh*)calloc(1, sizeof(ora_mesh));
    m->nv = nv;
    m->nc = nc;
    for (int a = 0; a < 3; ++a) m->period[a] = period[a];
    m->xyz = (double*)malloc(sizeof(double) * 3 * nv);
    m->tet = (int64_t*)malloc(sizeof(int64_t) * 4 * nc);
    m->shift = (int8_t*)malloc(sizeof(int8_t) * 12 * nc);
    memcpy(m->xyz, xyz, sizeof(double) * 3 * nv);
    memcpy(m->tet, tet, sizeof(int64_t) * 4 * nc);
    memcpy(m->shift, shift, sizeof(int8_t) * 12 * nc);
    for (int64_t i = 0; i < 4 * nc; ++i)
        if (tet[i] < 0 || tet[i] >= nv) {
            set_err(err, errlen, "vertex id out of range");
            ora_mesh_free(m);
            return NULL;
        }
    if (build_topology(m, err, errlen) || build_geometry(m, err, errlen)) {
        ora_mesh_free(m);
        return NULL;
    }
    build_stencils(m);
    return m;
}

int ora_mesh_set_boundary(ora_mesh* m, const int8_t* kind) {
    for (int64_t c = 0; c < m->nc; ++c)
        for (int f = 0; f < 4; ++f) {
            if (m->nbr[c * 4 + f] >= 0) continue;
            int8_t k = kind[c * 4 + f];
            if (k != ORA_BC_OPEN && k != ORA_BC_SLIP_WALL && k != ORA_BC_FIXED && k != ORA_BC_NOSLIP_WALL &&
                k != ORA_BC_ISOTHERMAL_WALL && k != ORA_BC_MOVING_WALL)
                return -1;
            m->bkind[m->csr_face[c * 4 + f]] = k;
        }
    build_wall_stencils(m);
    return 0;
}

void ora_mesh_set_fixed_state(ora_mesh* m, const double* W, const double* dW) {
    free(m->fixW);
    free(m->fixdW);
    m->fixW = (double*)malloc(sizeof(double) * 5 * m->nc);
    m->fixdW = (double*)malloc(sizeof(double) * 15 * m->nc);
    memcpy(m->fixW, W, sizeof(double) * 5 * m->nc);
    memcpy(m->fixdW, dW, sizeof(double) * 15 * m->nc);
}

void ora_mesh_free(ora_mesh* m) {
    if (!m) return;
    free(m->xyz); free(m->tet); free(m->shift);
    free(m->face_v); free(m->face_lr); free(m->nbr); free(m->nbr_shift);
    free(m->csr_face); free(m->csr_sign);
    free(m->vol); free(m->cen); free(m->mom2); free(m->dr);
    free(m->farea); free(m->fnorm); free(m->gp_l); free(m->gp_r);
    free(m->M1); free(m->M2); free(m->M2L); free(m->bkind); free(m->fixW); free(m->fixdW);
    free(m->MW1); free(m->MW2); free(m->wallc);
    free(m);
}

int64_t ora_mesh_nc(const ora_mesh* m) { return m->nc; }
int64_t ora_mesh_nf(const ora_mesh* m) { return m->nf; }
int64_t ora_mesh_n_singular(const ora_mesh* m) { return m->n_singular; }

void ora_mesh_topology(const ora_mesh* m, int64_t* face_v, int64_t* face_lr,
                       int64_t* nbr, int64_t* csr_face, int8_t* csr_sign) {
    if (face_v) memcpy(face_v, m->face_v, sizeof(int64_t) * 3 * m->nf);
    if (face_lr) memcpy(face_lr, m->face_lr, sizeof(int64_t) * 2 * m->nf);
    if (nbr) memcpy(nbr, m->nbr, sizeof(int64_t) * 4 * m->nc);
    if (csr_face) memcpy(csr_face, m->csr_face, sizeof(int64_t) * 4 * m->nc);
    if (csr_sign) memcpy(csr_sign, m->csr_sign, sizeof(int8_t) * 4 * m->nc);
}

void ora_mesh_geometry(const ora_mesh* m, double* vol, double* cen, double* mom2,
                       double* dr, double* farea, double* fnorm, double* gp_l,
                       double* gp_r) {
    if (vol) memcpy(vol, m->vol, sizeof(double) * m->nc);
    if (cen) memcpy(cen, m->cen, sizeof(double) * 3 * m->nc);
    if (mom2) memcpy(mom2, m->mom2, sizeof(double) * 6 * m->nc);
    if (dr) memcpy(dr, m->dr, sizeof(double) * m->nc);
    if (farea) memcpy(farea, m->farea, sizeof(double) * m->nf);
    if (fnorm) memcpy(fnorm, m->fnorm, sizeof(double) * 3 * m->nf);
    if (gp_l) memcpy(gp_l, m->gp_l, sizeof(double) * 9 * m->nf);
    if (gp_r) memcpy(gp_r, m->gp_r, sizeof(double) * 9 * m->nf);
}

void ora_mesh_stencils(const ora_mesh* m, double* M1, double* M2) {
    if (M1) memcpy(M1, m->M1, sizeof(double) * 12 * m->nc);
    if (M2) memcpy(M2, m->M2, sizeof(double) * 144 * m->nc);
}

/* ------------------------------------------------------------------------ */
/* reconstruction, Sec. 4                                                   */
/* ------------------------------------------------------------------------ */

/* A polynomial in "basis form" on cell c: v[0] is the coefficient of 1 and
 * v[1..9] those of the zero-mean basis p^k of Eq. base, in the order
 * x, y, z, xx, xy, xz, yy, yz, zz (coordinates relative to the centroid). */

/* gradient of a basis-form polynomial at X (relative to the centroid) */
static void basis_grad(const double v[10], const double X[3], double g[3]) {
    for (int l = 0; l < 3; ++l) {
        double s = v[1 + l];
        for (int q = 0; q < 6; ++q) {
            double dq = 0.0;
            if (QI[q] == l) dq += X[QJ[q]];
            if (QJ[q] == l) dq += X[QI[q]];
            s += v[4 + q] * dq;
        }
        g[l] = s;
    }
}

/* Smoothness indicator of Eq. smooth-indicator for a basis-form polynomial
 * of degree r (1 or 2), integrals by the 5-point volume rule. */
static double smoothness(const ora_mesh* m, int64_t c, const double v[10], int r) {
    double x[4][3], e[3][3];
    for (int k = 0; k < 4; ++k) cell_vertex(m, c, k, x[k]);
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 3; ++a) e[k][a] = x[k + 1][a] - x[0][a];
    double vol = m->vol[c];
    double jac = 6.0 * vol;
    double first = 0.0;
    for (int q = 0; q < 5; ++q) {
        double X[3], g[3];
        for (int a = 0; a < 3; ++a)
            X[a] = x[0][a] + VQ_P[q][0] * e[0][a] + VQ_P[q][1] * e[1][a] + VQ_P[q][2] * e[2][a] -
                   m->cen[c * 3 + a];
        basis_grad(v, X, g);
        first += VQ_W[q] * jac * (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    }
    double beta = pow(vol, 2.0 / 3.0 - 1.0) * first;
    if (r >= 2) {
        /* the six distinct second derivatives (READING: no multiplicity) */
        double second = 0.0;
        for (int q = 0; q < 6; ++q) {
            double dd = (QI[q] == QJ[q]) ? 2.0 * v[4 + q] : v[4 + q];
            second += vol * dd * dd;
        }
        beta += pow(vol, 4.0 / 3.0 - 1.0) * second;
    }
    return beta;
}

/* convert basis form to centroid-monomial form (subtract the basis means) */
static void basis_to_monomial(const ora_mesh* m, int64_t c, const double v[10], double out[10]) {
    double c0 = v[0];
    for (int q = 0; q < 6; ++q) c0 -= v[4 + q] * m->mom2[c * 6 + q];
    out[0] = c0;
    for (int k = 1; k < 10; ++k) out[k] = v[k];
}

static void monomial_eval(const double* P, const double X[3], double* val, double g[3]) {
    double q[6] = {X[0] * X[0], X[0] * X[1], X[0] * X[2], X[1] * X[1], X[1] * X[2], X[2] * X[2]};
    double s = P[0] + P[1] * X[0] + P[2] * X[1] + P[3] * X[2];
    for (int k = 0; k < 6; ++k) s += P[4 + k] * q[k];
    *val = s;
    if (g) {
        for (int l = 0; l < 3; ++l) {
            double t = P[1 + l];
            for (int k = 0; k < 6; ++k) {
                double dq = 0.0;
                if (QI[k] == l) dq += X[QJ[k]];
                if (QJ[k] == l) dq += X[QI[k]];
                t += P[4 + k] * dq;
            }
            g[l] = t;
        }
    }
}

/* beta_0 of the two-step reconstruction (Sec. 4.3, Eq. p0-non-linear-weight)
 * from the step-1 slopes b[j] of the cell's nn neighbours:
 *   beta_0,j = |Delta_0| |b_j|^2 with |Delta_0| = |Omega_0|^(2/3) (READING),
 *   sigma^1st = (mean over the neighbour pairs j > k of |beta_0,j - beta_0,k|)^(4/3)
 *   (READING: the mean over the existing pairs, 6 for an interior cell),
 *   omega^1st_j = 1 + sigma^1st / (eps + beta_0,j), normalised, and
 *   beta_0 = sum_j wbar^1st_j beta_0,j.
 * sigma1 and wbar1[nn] (each may be NULL) receive the intermediate values. */
static double weno_beta0(double vol, const double b[][3], int nn, double eps, double* sigma1,
                         double* wbar1) {
    double b0j[4];
    for (int j = 0; j < nn; ++j) b0j[j] = pow(vol, 2.0 / 3.0) * (b[j][0] * b[j][0] + b[j][1] * b[j][1] + b[j][2] * b[j][2]);
    double beta0 = 0.0, s1 = 0.0;
    if (nn > 0) {
        double sum = 0.0;
        int npair = 0;
        for (int j = 0; j < nn; ++j)
            for (int k = 0; k < j; ++k) { sum += fabs(b0j[j] - b0j[k]); ++npair; }
        s1 = npair ? pow(sum / npair, 4.0 / 3.0) : 0.0;
        double w1[4], ws = 0.0;
        for (int j = 0; j < nn; ++j) { w1[j] = 1.0 + s1 / (eps + b0j[j]); ws += w1[j]; }
        for (int j = 0; j < nn; ++j) {
            beta0 += w1[j] / ws * b0j[j];
            if (wbar1) wbar1[j] = w1[j] / ws;
        }
    }
    if (sigma1) *sigma1 = s1;
    return beta0;
}

/* normalised nonlinear weights (Sec. 4.2, Eq. non-linear-weight) of p_0, p_1
 * (order 2) or p_0, p_1, p_2 (order 3) into wbar[3]:
 *   sigma = |beta_1 - beta_0|^(4/3) (order 2) or
 *   (1/2 (|beta_2 - beta_1| + |beta_2 - beta_0|))^(4/3) (order 3),
 *   omega_m = gamma_m (1 + (sigma / (eps + beta_m))^2), wbar_m = omega_m / sum omega,
 * with gamma_1,1 : gamma_0,1 = 10 : 1 and gamma_2,2 : gamma_1,2 : gamma_0,2 =
 * 100 : 10 : 1 (READING of the Table 2 caption).  wbar[2] = 0 for order 2. */
static void weno_weights(int order, double eps, double beta0, double beta1, double beta2, double wbar[3]) {
    if (order == 2) {
        const double g11 = 10.0 / 11.0, g01 = 1.0 / 11.0;
        double sigma = pow(fabs(beta1 - beta0), 4.0 / 3.0);
        double w0 = g01 * (1.0 + pow(sigma / (eps + beta0), 2));
        double w1 = g11 * (1.0 + pow(sigma / (eps + beta1), 2));
        double ws = w0 + w1;
        wbar[0] = w0 / ws;
        wbar[1] = w1 / ws;
        wbar[2] = 0.0;
    } else {
        const double g22 = 100.0 / 111.0, g12 = 10.0 / 111.0, g02 = 1.0 / 111.0;
        double sigma = pow(0.5 * (fabs(beta2 - beta1) + fabs(beta2 - beta0)), 4.0 / 3.0);
        double w0 = g02 * (1.0 + pow(sigma / (eps + beta0), 2));
        double w1 = g12 * (1.0 + pow(sigma / (eps + beta1), 2));
        double w2 = g22 * (1.0 + pow(sigma / (eps + beta2), 2));
        double ws = w0 + w1 + w2;
        wbar[0] = w0 / ws;
        wbar[1] = w1 / ws;
        wbar[2] = w2 / ws;
    }
}

/* 1 where component q of cell c takes the Sec. 4.4 wall-constrained
 * stencils: a momentum component of a cell with a non-slip adiabatic wall
 * face whose constrained operators were built */
static int wall_constrained(const ora_mesh* m, const ora_params* p, int64_t c, int q) {
    return p->wall_constraint && m->wallc && m->wallc[c] && q >= 1 && q <= 3;
}

static void slopes_all(const ora_mesh* m, const ora_params* p, const double* W, double* b) {
    /* Reconstruction step 1 (Sec. 4.3; Sec. 4.4 at non-slip walls): P1
     * slopes of every cell */
    for (int64_t c = 0; c < m->nc; ++c)
        for (int q = 0; q < 5; ++q) {
            double dq[4];
            for (int f = 0; f < 4; ++f) {
                int64_t nb = m->nbr[c * 4 + f];
                dq[f] = nb >= 0 ? W[q * m->nc + nb] - W[q * m->nc + c] : 0.0;
            }
            int wall = wall_constrained(m, p, c, q);
            for (int i = 0; i < 3; ++i) {
                double s = 0.0;
                if (wall) {
                    for (int f = 0; f < 4; ++f) s += m->MW1[c * 15 + i * 5 + f] * dq[f];
                    s += m->MW1[c * 15 + i * 5 + 4] * W[q * m->nc + c];
                } else {
                    for (int f = 0; f < 4; ++f) s += m->M1[c * 12 + i * 4 + f] * dq[f];
                }
                b[(c * 5 + q) * 3 + i] = s;
            }
        }
}

int ora_reconstruct(const ora_mesh* m, const ora_params* p, const double* W,
                    const double* dW, double* poly, double* slopes_out,
                    int32_t* fallback) {
    const int64_t nc = m->nc;
    double* b = (double*)malloc(sizeof(double) * nc * 15);
    slopes_all(m, p, W, b);
    const double g22 = 100.0 / 111.0, g12 = 10.0 / 111.0, g02 = 1.0 / 111.0;
    const double g11 = 10.0 / 11.0, g01 = 1.0 / 11.0;
    const double eps = p->eps_weno;
    for (int64_t c = 0; c < nc; ++c) {
        double vol = m->vol[c];
        double R[5][10];
        for (int q = 0; q < 5; ++q) {
            double Q0 = W[q * nc + c];
            double data[16];
            for (int f = 0; f < 4; ++f) {
                int64_t nb = m->nbr[c * 4 + f];
                data[f] = nb >= 0 ? W[q * nc + nb] - Q0 : 0.0;
                for (int l = 0; l < 3; ++l)
                    data[4 + 3 * f + l] = nb >= 0 ? dW[(3 * q + l) * nc + nb] : 0.0;
            }
            double P0[10] = {Q0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
            double P1[10] = {Q0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
            double P2[10] = {Q0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
            for (int i = 0; i < 3; ++i) P1[1 + i] = b[(c * 5 + q) * 3 + i];
            int boundary = 0;
            for (int f = 0; f < 4; ++f) boundary |= m->nbr[c * 4 + f] < 0;
            if (wall_constrained(m, p, c, q)) {
                /* Sec. 4.4: P2 vanishing at the wall faces' Gauss points */
                for (int k = 0; k < 9; ++k) {
                    double s = m->MW2[c * 153 + k * 17 + 16] * Q0;
                    for (int j = 0; j < 16; ++j) s += m->MW2[c * 153 + k * 17 + j] * data[j];
                    P2[1 + k] = s;
                }
            } else if (boundary && !p->weno && p->order == 3) {
                /* Sec. 4.4: the first-order least-squares fit instead of P2 */
                for (int k = 0; k < 3; ++k) {
                    double s = 0.0;
                    for (int j = 0; j < 16; ++j) s += m->M2L[c * 48 + k * 16 + j] * data[j];
                    P2[1 + k] = s;
                }
            } else {
                for (int k = 0; k < 9; ++k) {
                    double s = 0.0;
                    for (int j = 0; j < 16; ++j) s += m->M2[c * 144 + k * 16 + j] * data[j];
                    P2[1 + k] = s;
                }
            }
            double Rb[10];
            if (!p->weno) {
                for (int k = 0; k < 10; ++k) Rb[k] = p->order == 2 ? P1[k] : P2[k];
            } else {
                /* beta_0 from the neighbours' step-1 slopes (Eq. p0-non-linear-weight) */
                double bj[4][3];
                int nn = 0;
                for (int f = 0; f < 4; ++f) {
                    int64_t nb = m->nbr[c * 4 + f];
                    if (nb < 0) continue;
                    for (int i = 0; i < 3; ++i) bj[nn][i] = b[(nb * 5 + q) * 3 + i];
                    ++nn;
                }
                double beta0 = weno_beta0(vol, bj, nn, eps, NULL, NULL);
                double beta1 = smoothness(m, c, P1, 1);
                double beta2 = p->order == 2 ? 0.0 : smoothness(m, c, P2, 2);
                double wbar[3];
                weno_weights(p->order, eps, beta0, beta1, beta2, wbar);
                double p0[10], p1[10], p2[10];
                for (int k = 0; k < 10; ++k) {
                    p0[k] = P0[k];
                    p1[k] = (P1[k] - g01 * P0[k]) / g11;
                }
                for (int k = 0; k < 10; ++k) p2[k] = (P2[k] - g12 * p1[k] - g02 * p0[k]) / g22;
                if (p->order == 2) {
                    for (int k = 0; k < 10; ++k) Rb[k] = wbar[1] * p1[k] + wbar[0] * p0[k];
                } else {
                    for (int k = 0; k < 10; ++k)
                        Rb[k] = wbar[2] * p2[k] + wbar[1] * p1[k] + wbar[0] * p0[k];
                }
            }
            basis_to_monomial(m, c, Rb, R[q]);
        }
        /* positivity (Sec. 4.2, READING: all 12 face Gauss points of the
         * cell; on failure the cell average is used for all components) */
        int bad = 0;
        for (int f = 0; f < 4 && !bad; ++f) {
            int64_t fi = m->csr_face[c * 4 + f];
            const double* gp = m->csr_sign[c * 4 + f] > 0 ? &m->gp_l[fi * 9] : &m->gp_r[fi * 9];
            for (int k = 0; k < 3 && !bad; ++k) {
                double v[5];
                for (int q = 0; q < 5; ++q) monomial_eval(R[q], &gp[k * 3], &v[q], NULL);
                double pr = (p->gamma - 1.0) * (v[4] - 0.5 * (v[1] * v[1] + v[2] * v[2] + v[3] * v[3]) / v[0]);
                if (!(v[0] > 0.0) || !(pr > 0.0)) bad = 1;
            }
        }
        if (bad)
            for (int q = 0; q < 5; ++q) {
                R[q][0] = W[q * nc + c];
                for (int k = 1; k < 10; ++k) R[q][k] = 0.0;
            }
        if (fallback) fallback[c] = bad;
        for (int q = 0; q < 5; ++q)
            for (int k = 0; k < 10; ++k) poly[(c * 5 + q) * 10 + k] = R[q][k];
    }
    if (slopes_out) memcpy(slopes_out, b, sizeof(double) * nc * 15);
    free(b);
    return 0;
}

double ora_smoothness(const ora_mesh* m, int64_t c, const double* v, int r) {
    return smoothness(m, c, v, r);
}

double ora_weno_beta0(double vol, const double* b, int nn, double eps, double* sigma1, double* wbar1) {
    double bj[4][3];
    for (int j = 0; j < nn && j < 4; ++j)
        for (int i = 0; i < 3; ++i) bj[j][i] = b[3 * j + i];
    return weno_beta0(vol, (const double(*)[3])bj, nn < 4 ? nn : 4, eps, sigma1, wbar1);
}

void ora_weno_weights(int order, double eps, double beta0, double beta1, double beta2, double* wbar) {
    weno_weights(order, eps, beta0, beta1, beta2, wbar);
}

/* ------------------------------------------------------------------------ */
/* velocity-space moments of a Maxwellian, Sec. 2.2                          */
/* ------------------------------------------------------------------------ */

/* sparse polynomial in (u1, u2, u3, xi^2) */
typedef struct { double c; int e[4]; } term;
typedef struct { int n; term t[64]; } poly;

static void poly_add_term(poly* p, double c, int e0, int e1, int e2, int e3) {
    if (p->n >= 64) { fprintf(stderr, "oracle poly overflow\n"); abort(); }
    term* t = &p->t[p->n++];
    t->c = c; t->e[0] = e0; t->e[1] = e1; t->e[2] = e2; t->e[3] = e3;
}

static poly poly_mul(const poly* a, const poly* b) {
    poly r;
    r.n = 0;
    for (int i = 0; i < a->n; ++i)
        for (int j = 0; j < b->n; ++j)
            poly_add_term(&r, a->t[i].c * b->t[j].c, a->t[i].e[0] + b->t[j].e[0],
                          a->t[i].e[1] + b->t[j].e[1], a->t[i].e[2] + b->t[j].e[2],
                          a->t[i].e[3] + b->t[j].e[3]);
    return r;
}

/* psi = (1, u1, u2, u3, (u1^2 + u2^2 + u3^2 + xi^2) / 2) */
static poly psi_poly(int a) {
    poly p;
    p.n = 0;
    switch (a) {
        case 0: poly_add_term(&p, 1.0, 0, 0, 0, 0); break;
        case 1: poly_add_term(&p, 1.0, 1, 0, 0, 0); break;
        case 2: poly_add_term(&p, 1.0, 0, 1, 0, 0); break;
        case 3: poly_add_term(&p, 1.0, 0, 0, 1, 0); break;
        default:
            poly_add_term(&p, 0.5, 2, 0, 0, 0);
            poly_add_term(&p, 0.5, 0, 2, 0, 0);
            poly_add_term(&p, 0.5, 0, 0, 2, 0);
            poly_add_term(&p, 0.5, 0, 0, 0, 1);
    }
    return p;
}

/* s = s_1 + s_2 u1 + s_3 u2 + s_4 u3 + s_5 (u^2 + xi^2)/2 */
static poly slope_poly(const double s[5]) {
    poly p;
    p.n = 0;
    poly_add_term(&p, s[0], 0, 0, 0, 0);
    poly_add_term(&p, s[1], 1, 0, 0, 0);
    poly_add_term(&p, s[2], 0, 1, 0, 0);
    poly_add_term(&p, s[3], 0, 0, 1, 0);
    poly_add_term(&p, 0.5 * s[4], 2, 0, 0, 0);
    poly_add_term(&p, 0.5 * s[4], 0, 2, 0, 0);
    poly_add_term(&p, 0.5 * s[4], 0, 0, 2, 0);
    poly_add_term(&p, 0.5 * s[4], 0, 0, 0, 1);
    return p;
}

static poly mono(int e0, int e1, int e2) {
    poly p;
    p.n = 0;
    poly_add_term(&p, 1.0, e0, e1, e2, 0);
    return p;
}

/* normalised moments <u1^k>, <u2^k>, <u3^k>, <xi^(2k)> of
 * g/rho = (lam/pi)^((K+3)/2) exp(-lam((u-U)^2 + xi^2)); half = +1 restricts
 * u1 > 0, -1 restricts u1 < 0, 0 is the whole space. */
typedef struct { double u[10], v[10], w[10], xi[4]; } mtab;

static void moment_1d(double* m, double U, double lam, int half) {
    if (half == 0) {
        m[0] = 1.0;
        m[1] = U;
    } else {
        double s = half > 0 ? 1.0 : -1.0;
        m[0] = 0.5 * erfc(-s * sqrt(lam) * U);
        m[1] = U * m[0] + s * 0.5 * exp(-lam * U * U) / sqrt(ORA_PI * lam);
    }
    for (int k = 0; k + 2 < 10; ++k) m[k + 2] = U * m[k + 1] + (k + 1) / (2.0 * lam) * m[k];
}

static void mtab_build(mtab* t, const double U[3], double lam, double K, int half) {
    moment_1d(t->u, U[0], lam, half);
    moment_1d(t->v, U[1], lam, 0);
    moment_1d(t->w, U[2], lam, 0);
    t->xi[0] = 1.0;
    t->xi[1] = K / (2.0 * lam);
    t->xi[2] = (K * K + 2.0 * K) / (4.0 * lam * lam);
    t->xi[3] = K * (K + 2.0) * (K + 4.0) / (8.0 * lam * lam * lam);
}

static double poly_moment(const mtab* t, const poly* p) {
    double s = 0.0;
    for (int i = 0; i < p->n; ++i) {
        const term* q = &p->t[i];
        if (q->e[0] > 9 || q->e[1] > 9 || q->e[2] > 9 || q->e[3] > 3) {
            fprintf(stderr, "oracle moment order overflow\n");
            abort();
        }
        s += q->c * t->u[q->e[0]] * t->v[q->e[1]] * t->w[q->e[2]] * t->xi[q->e[3]];
    }
    return s;
}

/* out[a] = < psi_a * p > */
static void psi_moments(const mtab* t, const poly* p, double out[5]) {
    for (int a = 0; a < 5; ++a) {
        poly ps = psi_poly(a);
        poly pr = poly_mul(&ps, p);
        out[a] = poly_moment(t, &pr);
    }
}

/* micro-slope solve (Eq. co): < s psi > = rhs, by a direct 5x5 solve */
static void micro_slope(const mtab* full, const double rhs[5], double s[5]) {
    double M[25], B[5];
    for (int a = 0; a < 5; ++a) {
        poly pa = psi_poly(a);
        for (int b = 0; b < 5; ++b) {
            poly pb = psi_poly(b);
            poly pr = poly_mul(&pa, &pb);
            M[a * 5 + b] = poly_moment(full, &pr);
        }
        B[a] = rhs[a];
    }
    gauss_solve(5, 1, M, B, NULL, NULL);
    for (int a = 0; a < 5; ++a) s[a] = B[a];
}

typedef struct { double rho, U[3], lam, p; } prim;

static prim to_prim(const double W[5], double gamma) {
    prim r;
    r.rho = W[0];
    for (int i = 0; i < 3; ++i) r.U[i] = W[1 + i] / W[0];
    double ke = 0.5 * r.rho * (r.U[0] * r.U[0] + r.U[1] * r.U[1] + r.U[2] * r.U[2]);
    r.p = (gamma - 1.0) * (W[4] - ke);
    r.lam = r.rho / (2.0 * r.p);
    return r;
}

/* <psi * (sum_i a_i u_i) * extra> on table t, extra a monomial */
static void grad_term(const mtab* t, const double a[3][5], int e0, int e1, int e2, double out[5]) {
    for (int k = 0; k < 5; ++k) out[k] = 0.0;
    for (int i = 0; i < 3; ++i) {
        poly s = slope_poly(a[i]);
        poly ui = mono(e0 + (i == 0), e1 + (i == 1), e2 + (i == 2));
        poly pr = poly_mul(&s, &ui);
        double o[5];
        psi_moments(t, &pr, o);
        for (int k = 0; k < 5; ++k) out[k] += o[k];
    }
}

/* the slopes a_{x_i} (i = 1..3) and A of a Maxwellian with derivatives dW */
static void slopes_of_state(const mtab* full, const prim* st, const double dW[3][5],
                            double a[3][5], double A[5]) {
    for (int i = 0; i < 3; ++i) {
        double rhs[5];
        for (int k = 0; k < 5; ++k) rhs[k] = dW[i][k] / st->rho;
        micro_slope(full, rhs, a[i]);
    }
    double r[5];
    grad_term(full, a, 0, 0, 0, r);
    for (int k = 0; k < 5; ++k) r[k] = -r[k];
    micro_slope(full, r, A);
}

/* Pr fix of one interval's flux F given its state integral IW = int psi f:
 * F_E += prf q, q = F_E - U.F_m + |U|^2/2 F_rho - U1 (IW_E - U.IW_m + |U|^2/2 IW_rho) */
static void heat_flux_fix(double prf, const double U[3], const double IW[5], double F[5]) {
    double uu = 0.5 * (U[0] * U[0] + U[1] * U[1] + U[2] * U[2]);
    double qf = F[4] - (U[0] * F[1] + U[1] * F[2] + U[2] * F[3]) + uu * F[0];
    double qw = IW[4] - (U[0] * IW[1] + U[1] * IW[2] + U[2] * IW[3]) + uu * IW[0];
    F[4] += prf * (qf - U[0] * qw);
}

void ora_gp_flux(const ora_params* p, const double* Wl, const double* dWl_,
                 const double* Wr, const double* dWr_, double dt, double* Fh,
                 double* F, double* W0, double* Wdt) {
    const double gamma = p->gamma;
    const double K = (5.0 - 3.0 * gamma) / (gamma - 1.0);
    double dWl[3][5], dWr[3][5];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 5; ++k) { dWl[i][k] = dWl_[i * 5 + k]; dWr[i][k] = dWr_[i * 5 + k]; }
    prim L = to_prim(Wl, gamma), R = to_prim(Wr, gamma);
    mtab fl, fr, hl, hr;
    mtab_build(&fl, L.U, L.lam, K, 0);
    mtab_build(&fr, R.U, R.lam, K, 0);
    mtab_build(&hl, L.U, L.lam, K, +1);
    mtab_build(&hr, R.U, R.lam, K, -1);
    double al[3][5], Al[5], ar[3][5], Ar[5];
    slopes_of_state(&fl, &L, dWl, al, Al);
    slopes_of_state(&fr, &R, dWr, ar, Ar);

    /* equilibrium state at the interface by kinetic weighting (Eq. new-equ-part) */
    poly one = mono(0, 0, 0);
    double Wc[5], ml[5], mr[5];
    psi_moments(&hl, &one, ml);
    psi_moments(&hr, &one, mr);
    for (int k = 0; k < 5; ++k) Wc[k] = L.rho * ml[k] + R.rho * mr[k];
    double dWc[3][5];
    for (int i = 0; i < 3; ++i) {
        poly sl = slope_poly(al[i]), sr = slope_poly(ar[i]);
        psi_moments(&hl, &sl, ml);
        psi_moments(&hr, &sr, mr);
        for (int k = 0; k < 5; ++k) dWc[i][k] = L.rho * ml[k] + R.rho * mr[k];
    }
    prim C = to_prim(Wc, gamma);
    mtab fc;
    mtab_build(&fc, C.U, C.lam, K, 0);
    double ac[3][5], Ac[5];
    slopes_of_state(&fc, &C, dWc, ac, Ac);

    /* collision times (Sec. 2.2) */
    double tau = p->viscous ? p->mu / C.p : 0.0;
    double jump = fabs((L.p - R.p) / (L.p + R.p)) * dt;
    double tau_n = (p->viscous ? p->mu / C.p : p->tau_eps * dt) + p->tau_c * jump;

    /* moment vectors needed by Eq. 2nd-flux, with and without u1 */
    double c_f[5], c_fa[5], c_fA[5], c_w[5], c_wa[5], c_wA[5];
    double l_f[5], l_fa[5], l_fA[5], l_w[5], l_wa[5], l_wA[5];
    double r_f[5], r_fa[5], r_fA[5], r_w[5], r_wa[5], r_wA[5];
    poly u1 = mono(1, 0, 0);
    poly pAc = slope_poly(Ac), pAl = slope_poly(Al), pAr = slope_poly(Ar);
    poly u1Ac = poly_mul(&u1, &pAc), u1Al = poly_mul(&u1, &pAl), u1Ar = poly_mul(&u1, &pAr);
    psi_moments(&fc, &u1, c_f);
    grad_term(&fc, ac, 1, 0, 0, c_fa);
    psi_moments(&fc, &u1Ac, c_fA);
    psi_moments(&fc, &one, c_w);
    grad_term(&fc, ac, 0, 0, 0, c_wa);
    psi_moments(&fc, &pAc, c_wA);
    psi_moments(&hl, &u1, l_f);
    grad_term(&hl, al, 1, 0, 0, l_fa);
    psi_moments(&hl, &u1Al, l_fA);
    psi_moments(&hl, &one, l_w);
    grad_term(&hl, al, 0, 0, 0, l_wa);
    psi_moments(&hl, &pAl, l_wA);
    psi_moments(&hr, &u1, r_f);
    grad_term(&hr, ar, 1, 0, 0, r_fa);
    psi_moments(&hr, &u1Ar, r_fA);
    psi_moments(&hr, &one, r_w);
    grad_term(&hr, ar, 0, 0, 0, r_wa);
    psi_moments(&hr, &pAr, r_wA);

    /* Pr fix (viscous, Pr != 1): the energy flux over [0, d] gains
     * (1/Pr - 1) q, q = int_0^d int (u1 - U1) (|u - U|^2 + xi^2)/2 f, U the
     * interface equilibrium velocity.  The paper names no formula (BGK has
     * Pr = 1, Sec. 2); READING: the heat-flux correction of the gas-kinetic
     * Navier-Stokes solver, applied to the time-integrated flux.  Since
     * (u1 - U1)|c|^2/2 = u1 eps - u1 U.u + u1 |U|^2/2 - U1 (eps - U.u + |U|^2/2),
     * q follows from the interval's flux and its state integral IW. */
    const double prf = p->viscous ? 1.0 / p->prandtl - 1.0 : 0.0;
    double IW[2][5];

    if (p->smooth_flux) {
        /* Eq. 2nd-smooth-flux: f = g^c - tau (a^c.u + A^c) g^c + A^c g^c t */
        for (int h = 0; h < 2; ++h) {
            double d = h == 0 ? 0.5 * dt : dt;
            double* out = h == 0 ? Fh : F;
            for (int k = 0; k < 5; ++k) {
                out[k] = C.rho * (d * c_f[k] - tau * d * (c_fa[k] + c_fA[k]) + 0.5 * d * d * c_fA[k]);
                IW[h][k] = C.rho * (d * c_w[k] - tau * d * (c_wa[k] + c_wA[k]) + 0.5 * d * d * c_wA[k]);
            }
            if (prf != 0.0) heat_flux_fix(prf, C.U, IW[h], out);
        }
        for (int h = 0; h < 2; ++h) {
            double t = h == 0 ? 0.0 : dt;
            double* out = h == 0 ? W0 : Wdt;
            for (int k = 0; k < 5; ++k)
                out[k] = C.rho * (c_w[k] - tau * (c_wa[k] + c_wA[k]) + t * c_wA[k]);
        }
        return;
    }

    /* Eq. 2nd-flux integrated over [0, d]: hydrodynamic factors C1..C3 and
     * the kinetic factors e and t e, with the exponentials in tau_n */
    for (int h = 0; h < 2; ++h) {
        double d = h == 0 ? 0.5 * dt : dt;
        double E = exp(-d / tau_n);
        double k0 = tau_n * (1.0 - E);                 /* int e */
        double k1 = tau_n * tau_n * (1.0 - E) - tau_n * d * E; /* int t e */
        double q1 = d - k0;                            /* int C1 */
        double q2 = k1 + tau * k0 - tau * d;           /* int C2 */
        double q3 = 0.5 * d * d - tau * d + tau * k0;  /* int C3 */
        double* out = h == 0 ? Fh : F;
        for (int k = 0; k < 5; ++k) {
            out[k] = C.rho * (q1 * c_f[k] + q2 * c_fa[k] + q3 * c_fA[k]) +
                     L.rho * (k0 * l_f[k] - (tau * k0 + k1) * l_fa[k] - tau * k0 * l_fA[k]) +
                     R.rho * (k0 * r_f[k] - (tau * k0 + k1) * r_fa[k] - tau * k0 * r_fA[k]);
            IW[h][k] = C.rho * (q1 * c_w[k] + q2 * c_wa[k] + q3 * c_wA[k]) +
                       L.rho * (k0 * l_w[k] - (tau * k0 + k1) * l_wa[k] - tau * k0 * l_wA[k]) +
                       R.rho * (k0 * r_w[k] - (tau * k0 + k1) * r_wa[k] - tau * k0 * r_wA[k]);
        }
        if (prf != 0.0) heat_flux_fix(prf, C.U, IW[h], out);
    }
    /* point values of f at t = 0 and t = dt */
    for (int h = 0; h < 2; ++h) {
        double t = h == 0 ? 0.0 : dt;
        double e = exp(-t / tau_n);
        double C1 = 1.0 - e, C2 = (t + tau) * e - tau, C3 = t - tau + tau * e;
        double* out = h == 0 ? W0 : Wdt;
        for (int k = 0; k < 5; ++k)
            out[k] = C.rho * (C1 * c_w[k] + C2 * c_wa[k] + C3 * c_wA[k]) +
                     L.rho * (e * l_w[k] - (tau + t) * e * l_wa[k] - tau * e * l_wA[k]) +
                     R.rho * (e * r_w[k] - (tau + t) * e * r_wa[k] - tau * e * r_wA[k]);
    }
}

/* ------------------------------------------------------------------------ */
/* local frame, Sec. 2.1                                                    */
/* ------------------------------------------------------------------------ */

static void frame_matrix(const double n[3], double T[5][5]) {
    memset(T, 0, sizeof(double) * 25);
    T[0][0] = 1.0;
    T[4][4] = 1.0;
    if (n[0] == -1.0) {
        T[1][1] = -1.0; T[2][2] = -1.0; T[3][3] = 1.0;
        return;
    }
    double n1 = n[0], n2 = n[1], n3 = n[2];
    T[1][1] = n1; T[1][2] = n2; T[1][3] = n3;
    T[2][1] = -n2; T[2][2] = n1 + n3 * n3 / (1.0 + n1); T[2][3] = -n2 * n3 / (1.0 + n1);
    T[3][1] = -n3; T[3][2] = -n2 * n3 / (1.0 + n1); T[3][3] = 1.0 - n3 * n3 / (1.0 + n1);
}

/* ------------------------------------------------------------------------ */
/* stage assembly, Sec. 3                                                   */
/* ------------------------------------------------------------------------ */

/* Stage 1 uses F(t_n) dt + F_t dt^2 / 8 ... folded: with the linear fit of
 * Eq. linear-system, dt/2 L + dt^2/8 L_t involves only Fh, and
 * dt L + dt^2/6 L_t involves 8/3 Fh - 1/3 F; the stage-2 term
 * dt^2/3 L_t(W*) involves 4/3 (F* - 2 Fh*). */
static void fit_flux(const double* Fh, const double* F, double dt, int n, double* F0, double* Ft) {
    for (int k = 0; k < n; ++k) {
        F0[k] = (4.0 * Fh[k] - F[k]) / dt;
        Ft[k] = 4.0 * (F[k] - 2.0 * Fh[k]) / (dt * dt);
    }
}
static void stage1_terms(const double* Fh, const double* F, double dt, int n, double* half, double* full) {
    /* half = dt/2 F0 + dt^2/8 Ft ; full = dt F0 + dt^2/6 Ft  (Eq. s2o4) */
    double F0[5], Ft[5];
    fit_flux(Fh, F, dt, n, F0, Ft);
    for (int k = 0; k < n; ++k) {
        half[k] = 0.5 * dt * F0[k] + dt * dt / 8.0 * Ft[k];
        full[k] = dt * F0[k] + dt * dt / 6.0 * Ft[k];
    }
}
static void stage2_terms(const double* Fh, const double* F, double dt, int n, double* out) {
    /* out = dt^2/6 * 2 * Ft(W*)  (Eq. s2o4) */
    double F0[5], Ft[5];
    fit_flux(Fh, F, dt, n, F0, Ft);
    for (int k = 0; k < n; ++k) out[k] = dt * dt / 3.0 * Ft[k];
}

double ora_s2o4_linear_ode(double z) {
    /* y' = lam y with lam = z / dt, dt = 1, |Omega| = 1, outward flux
     * F = -lam y.  As in the kinetic solver, the flux over a stage is linear
     * in time with the exact instantaneous derivative, F(t) = F0 + t Ft with
     * F0 = -lam y, Ft = -lam^2 y, so its integral over [0, d] is
     * F0 d + Ft d^2 / 2; the linear fit of Eq. linear-system then recovers
     * F0 and Ft and Eq. s2o4 must reproduce exp(z) to fourth order. */
    double dt = 1.0, lam = z / dt;
    double y0 = 1.0;
    double Fh = -y0 * (lam * 0.5 * dt + lam * lam * 0.125 * dt * dt);
    double F = -y0 * (lam * dt + lam * lam * 0.5 * dt * dt);
    double half, full;
    stage1_terms(&Fh, &F, dt, 1, &half, &full);
    double ys = y0 - half;
    double Fhs = -ys * (lam * 0.5 * dt + lam * lam * 0.125 * dt * dt);
    double Fs = -ys * (lam * dt + lam * lam * 0.5 * dt * dt);
    double two;
    stage2_terms(&Fhs, &Fs, dt, 1, &two);
    return (y0 - (full + two)) / y0;
}

/* ------------------------------------------------------------------------ */
/* face records                                                             */
/* ------------------------------------------------------------------------ */

/* Sec. 4.4, non-slip isothermal wall at rest, in the face frame (gas
 * constant R = 1, T = p / rho), following the paper's steps: the ghost keeps
 * the pressure, reverses the velocity and takes T = 2 T_wall - T; for its
 * derivatives, the interior's primitive derivatives (dU_i from d(rho U_i)
 * and d rho; dp from d(rho E), d rho and dQ with Q = |U|^2 / 2; dT from dp
 * and d rho) are taken with dU and dT kept and dp reversed, then turned
 * back into conservative derivatives of the ghost (d rho from dp and dT,
 * d(rho U_i), d(rho E)). */
static void isothermal_ghost(double W[5], double g[3][5], double gamma, double Tw) {
    double rho = W[0], U[3], Q = 0.0;
    for (int i = 0; i < 3; ++i) { U[i] = W[1 + i] / rho; Q += 0.5 * U[i] * U[i]; }
    double p = (gamma - 1.0) * (W[4] - rho * Q);
    double Tr = p / rho;
    double Tl = 2.0 * Tw - Tr;
    double rl = p / Tl;
    double Ul[3] = {-U[0], -U[1], -U[2]};
    double Wl[5] = {rl, rl * Ul[0], rl * Ul[1], rl * Ul[2], p / (gamma - 1.0) + rl * Q};
    for (int j = 0; j < 3; ++j) {
        /* interior primitive derivatives along x_j */
        double dU[3], dQ = 0.0;
        for (int i = 0; i < 3; ++i) { dU[i] = (g[j][1 + i] - g[j][0] * U[i]) / rho; dQ += U[i] * dU[i]; }
        double dp = (gamma - 1.0) * (g[j][4] - g[j][0] * Q - dQ * rho);
        double dT = (dp - g[j][0] * Tr) / rho;
        /* the ghost's: dU, dT kept, dp reversed */
        double dpl = -dp, dTl = dT, dQl = 0.0;
        for (int i = 0; i < 3; ++i) dQl += dU[i] * Ul[i];
        double drl = (dpl - dTl * rl) / Tl;
        g[j][0] = drl;
        for (int i = 0; i < 3; ++i) g[j][1 + i] = drl * Ul[i] + dU[i] * rl;
        g[j][4] = drl * Q + dQl * rl + dpl / (gamma - 1.0);
    }
    for (int k = 0; k < 5; ++k) W[k] = Wl[k];
}

/* Non-slip adiabatic wall moving along itself with velocity Uw (face frame;
 * the paper prints no ghost for it).  READING: the at-rest rules written in
 * primitive variables and shifted to the wall's frame: the ghost has the
 * interior density and pressure and the velocity 2 Uw - U; the velocity
 * derivatives are kept, the density and pressure derivatives reversed (at
 * Uw = 0 exactly the non-slip adiabatic ghost). */
static void moving_ghost(double W[5], double g[3][5], double gamma, const double Uw[3]) {
    double rho = W[0], U[3], Ul[3], Q = 0.0, Ql = 0.0;
    for (int i = 0; i < 3; ++i) {
        U[i] = W[1 + i] / rho;
        Ul[i] = 2.0 * Uw[i] - U[i];
        Q += 0.5 * U[i] * U[i];
        Ql += 0.5 * Ul[i] * Ul[i];
    }
    double p = (gamma - 1.0) * (W[4] - rho * Q);
    for (int j = 0; j < 3; ++j) {
        double dU[3], dQ = 0.0;
        for (int i = 0; i < 3; ++i) { dU[i] = (g[j][1 + i] - g[j][0] * U[i]) / rho; dQ += U[i] * dU[i]; }
        double dp = (gamma - 1.0) * (g[j][4] - g[j][0] * Q - dQ * rho);
        /* ghost: d rho and dp reversed, dU kept */
        double drho = -g[j][0], dpl = -dp, dQl = 0.0;
        for (int i = 0; i < 3; ++i) dQl += Ul[i] * dU[i];
        g[j][0] = drho;
        for (int i = 0; i < 3; ++i) g[j][1 + i] = drho * Ul[i] + rho * dU[i];
        g[j][4] = dpl / (gamma - 1.0) + drho * Ql + rho * dQl;
    }
    W[0] = rho;
    for (int i = 0; i < 3; ++i) W[1 + i] = rho * Ul[i];
    W[4] = p / (gamma - 1.0) + rho * Ql;
}

int ora_face_records(const ora_mesh* m, const ora_params* p, const double* W,
                     const double* dW, double dt, int stage, double* rec) {
    const int64_t nc = m->nc;
    const int nrec = stage == 1 ? 40 : 20;
    if (!m->fixW)
        for (int64_t f = 0; f < m->nf; ++f)
            if ((m->face_lr[f * 2] < 0 || m->face_lr[f * 2 + 1] < 0) && m->bkind[f] == ORA_BC_FIXED)
                return -1; /* a fixed boundary without its state */
    double* poly_ = (double*)malloc(sizeof(double) * nc * 50);
    ora_reconstruct(m, p, W, dW, poly_, NULL, NULL);
    for (int64_t f = 0; f < m->nf; ++f) {
        double* r = &rec[f * nrec];
        for (int k = 0; k < nrec; ++k) r[k] = 0.0;
        int64_t cl = m->face_lr[f * 2], cr = m->face_lr[f * 2 + 1];
        const double* n = &m->fnorm[f * 3];
        double T[5][5];
        frame_matrix(n, T);
        double w = m->farea[f] / 3.0; /* READING: weights carry the area */
        for (int k = 0; k < 3; ++k) {
            double WL[5], gL[3][5], WR[5], gR[3][5];
            for (int side = 0; side < 2; ++side) {
                int64_t c = side == 0 ? cl : cr;
                if (c < 0) continue;
                const double* X = side == 0 ? &m->gp_l[f * 9 + k * 3] : &m->gp_r[f * 9 + k * 3];
                double* Wv = side == 0 ? WL : WR;
                double (*g)[5] = side == 0 ? gL : gR;
                for (int q = 0; q < 5; ++q) {
                    double gg[3];
                    monomial_eval(&poly_[(c * 5 + q) * 10], X, &Wv[q], gg);
                    for (int i = 0; i < 3; ++i) g[i][q] = gg[i];
                }
            }
            /* READING: the paper leaves open (outflow) boundaries unspecified.
             * The ghost side of an open boundary face is the interior cell's
             * average with zero gradient (zeroth-order extrapolation).  Copying
             * the interior Gauss-point state, with or without its gradient,
             * amplifies rounding noise without bound next to the boundary. */
            for (int side = 0; side < 2; ++side) {
                int64_t inner = side == 0 ? cr : cl;
                if ((side == 0 ? cl : cr) >= 0 || m->bkind[f] != ORA_BC_OPEN) continue;
                double* Wg = side == 0 ? WL : WR;
                double (*gg)[5] = side == 0 ? gL : gR;
                for (int q = 0; q < 5; ++q) {
                    Wg[q] = W[q * nc + inner];
                    gg[0][q] = gg[1][q] = gg[2][q] = 0.0;
                }
            }
            /* a fixed boundary's ghost is the fixed state of the interior
             * cell (its average and gradient) extended linearly to the
             * Gauss point, with that gradient: a prescribed profile carried
             * past the boundary (the Shu-Osher right end, Sec. 5.2; a far
             * field, Sec. 5) */
            for (int side = 0; side < 2; ++side) {
                int64_t inner = side == 0 ? cr : cl;
                if ((side == 0 ? cl : cr) >= 0 || m->bkind[f] != ORA_BC_FIXED) continue;
                const double* X = side == 0 ? &m->gp_r[f * 9 + k * 3] : &m->gp_l[f * 9 + k * 3];
                double* Wg = side == 0 ? WL : WR;
                double (*gg)[5] = side == 0 ? gL : gR;
                for (int q = 0; q < 5; ++q) {
                    Wg[q] = m->fixW[q * nc + inner];
                    for (int i = 0; i < 3; ++i) {
                        gg[i][q] = m->fixdW[(3 * q + i) * nc + inner];
                        Wg[q] += gg[i][q] * X[i];
                    }
                }
            }
            /* a slip wall's ghost is built from the interior Gauss-point
             * state after the rotation (below); give the missing side the
             * interior values so the rotation leaves them defined */
            int wall = (cl < 0 || cr < 0) &&
                       (m->bkind[f] == ORA_BC_SLIP_WALL || m->bkind[f] == ORA_BC_NOSLIP_WALL ||
                        m->bkind[f] == ORA_BC_ISOTHERMAL_WALL || m->bkind[f] == ORA_BC_MOVING_WALL);
            if (wall) {
                if (cl < 0) {
                    memcpy(WL, WR, sizeof WL);
                    memcpy(gL, gR, sizeof gL);
                } else {
                    memcpy(WR, WL, sizeof WR);
                    memcpy(gR, gL, sizeof gR);
                }
            }
            /* rotate into the local frame: components by T, directions by
             * its velocity block */
            double tWL[5], tWR[5], tgL[3][5], tgR[3][5];
            for (int a = 0; a < 5; ++a) {
                tWL[a] = 0.0; tWR[a] = 0.0;
                for (int b = 0; b < 5; ++b) { tWL[a] += T[a][b] * WL[b]; tWR[a] += T[a][b] * WR[b]; }
            }
            for (int j = 0; j < 3; ++j)
                for (int a = 0; a < 5; ++a) {
                    double sl = 0.0, sr = 0.0;
                    for (int i = 0; i < 3; ++i)
                        for (int b = 0; b < 5; ++b) {
                            sl += T[1 + j][1 + i] * T[a][b] * gL[i][b];
                            sr += T[1 + j][1 + i] * T[a][b] * gR[i][b];
                        }
                    tgL[j][a] = sl;
                    tgR[j][a] = sr;
                }
            if (wall) {
                /* Sec. 4.4, slip wall, in the face frame (x1 along n): the
                 * ghost copies rho, rho U2, rho U3, rho E and reverses rho U1;
                 * of the x1-derivatives only that of rho U1 is kept, the
                 * others change sign; of the x2- and x3-derivatives only
                 * those of rho U1 change sign. */
                double* gW = cl < 0 ? tWL : tWR;
                double (*gg)[5] = cl < 0 ? tgL : tgR;
                if (m->bkind[f] == ORA_BC_SLIP_WALL) {
                    gW[1] = -gW[1];
                    for (int a = 0; a < 5; ++a)
                        if (a != 1) gg[0][a] = -gg[0][a];
                    gg[1][1] = -gg[1][1];
                    gg[2][1] = -gg[2][1];
                } else if (m->bkind[f] == ORA_BC_ISOTHERMAL_WALL) {
                    isothermal_ghost(gW, gg, p->gamma, p->wall_temperature);
                } else if (m->bkind[f] == ORA_BC_MOVING_WALL) {
                    double Uw[3];
                    for (int j = 0; j < 3; ++j)
                        Uw[j] = T[1 + j][1] * p->wall_velocity[0] + T[1 + j][2] * p->wall_velocity[1] +
                                T[1 + j][3] * p->wall_velocity[2];
                    moving_ghost(gW, gg, p->gamma, Uw);
                } else {
                    /* Sec. 4.4, non-slip adiabatic wall (at rest): the ghost
                     * keeps rho and rho E and reverses all three momenta;
                     * every derivative of the momenta is kept, every
                     * derivative of rho and of rho E changes sign. */
                    for (int a = 1; a <= 3; ++a) gW[a] = -gW[a];
                    for (int j = 0; j < 3; ++j) {
                        gg[j][0] = -gg[j][0];
                        gg[j][4] = -gg[j][4];
                    }
                }
            }
            double tFh[5], tF[5], tW0[5], tWdt[5];
            ora_gp_flux(p, tWL, &tgL[0][0], tWR, &tgR[0][0], dt, tFh, tF, tW0, tWdt);
            /* back to the global frame with T^-1 = T^T (Eq. flux-local-to-global) */
            double Fhv[5], Fv[5], W0v[5], Wdv[5];
            for (int a = 0; a < 5; ++a) {
                Fhv[a] = Fv[a] = W0v[a] = Wdv[a] = 0.0;
                for (int b = 0; b < 5; ++b) {
                    Fhv[a] += T[b][a] * tFh[b];
                    Fv[a] += T[b][a] * tF[b];
                    W0v[a] += T[b][a] * tW0[b];
                    Wdv[a] += T[b][a] * tWdt[b];
                }
            }
            if (stage == 1) {
                double half[5], full[5];
                stage1_terms(Fhv, Fv, dt, 5, half, full);
                for (int q = 0; q < 5; ++q) {
                    r[q] += w * half[q];
                    r[5 + q] += w * full[q];
                    for (int i = 0; i < 3; ++i) {
                        /* f* = f^n + dt/2 f_t^n (Eq. step-du) */
                        double Wstar = W0v[q] + 0.5 * dt * (Wdv[q] - W0v[q]) / dt;
                        r[10 + 3 * q + i] += w * Wstar * n[i];
                        r[25 + 3 * q + i] += w * W0v[q] * n[i];
                    }
                }
            } else {
                double two[5];
                stage2_terms(Fhv, Fv, dt, 5, two);
                for (int q = 0; q < 5; ++q) {
                    r[q] += w * two[q];
                    for (int i = 0; i < 3; ++i)
                        /* f^{n+1} = f^n + dt f_t^* (Eq. step-du) */
                        r[5 + 3 * q + i] += w * dt * ((Wdv[q] - W0v[q]) / dt) * n[i];
                }
            }
        }
    }
    free(poly_);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* time step (Eq. time-step) and the two-stage step (Eq. s2o4)               */
/* ------------------------------------------------------------------------ */

double ora_timestep(const ora_mesh* m, const ora_params* p, const double* W) {
    double dt = INFINITY;
    for (int64_t c = 0; c < m->nc; ++c) {
        double Wc[5];
        for (int q = 0; q < 5; ++q) Wc[q] = W[q * m->nc + c];
        prim s = to_prim(Wc, p->gamma);
        double U = sqrt(s.U[0] * s.U[0] + s.U[1] * s.U[1] + s.U[2] * s.U[2]);
        double a = sqrt(p->gamma * s.p / s.rho);
        double d = m->dr[c] / (U + a);
        if (p->viscous && p->mu > 0.0) {
            double nu = p->mu / s.rho;
            double dv = m->dr[c] * m->dr[c] / (3.0 * nu);
            if (dv < d) d = dv;
        }
        if (p->cfl * d < dt) dt = p->cfl * d;
    }
    return dt;
}

int ora_step(const ora_mesh* m, const ora_params* p, double* W, double* dW,
             double dt, double* dt_used) {
    const int64_t nc = m->nc, nf = m->nf;
    if (!(dt > 0.0)) dt = ora_timestep(m, p, W);
    if (dt_used) *dt_used = dt;
    double* rec1 = (double*)malloc(sizeof(double) * nf * 40);
    double* rec2 = (double*)malloc(sizeof(double) * nf * 20);
    double* Ws = (double*)calloc((size_t)nc * 5, sizeof(double));
    double* dWs = (double*)calloc((size_t)nc * 15, sizeof(double));
    double* S = (double*)malloc(sizeof(double) * nc * 5);
    double* G = (double*)malloc(sizeof(double) * nc * 15);
    if (ora_face_records(m, p, W, dW, dt, 1, rec1) != 0) {
        free(rec1); free(rec2); free(Ws); free(dWs); free(S); free(G);
        return -1;
    }
    for (int64_t c = 0; c < nc; ++c) {
        double fh[5] = {0}, s[5] = {0}, gs[15] = {0}, g0[15] = {0};
        for (int f = 0; f < 4; ++f) {
            int64_t fi = m->csr_face[c * 4 + f];
            double sg = m->csr_sign[c * 4 + f];
            for (int q = 0; q < 5; ++q) { fh[q] += sg * rec1[fi * 40 + q]; s[q] += sg * rec1[fi * 40 + 5 + q]; }
            for (int q = 0; q < 15; ++q) { gs[q] += sg * rec1[fi * 40 + 10 + q]; g0[q] += sg * rec1[fi * 40 + 25 + q]; }
        }
        for (int q = 0; q < 5; ++q) {
            Ws[q * nc + c] = W[q * nc + c] - fh[q] / m->vol[c];
            S[c * 5 + q] = s[q];
        }
        for (int q = 0; q < 15; ++q) {
            dWs[q * nc + c] = gs[q] / m->vol[c]; /* Eq. gauss-formula at t* */
            G[c * 15 + q] = g0[q];
        }
    }
    ora_face_records(m, p, Ws, dWs, dt, 2, rec2);
    for (int64_t c = 0; c < nc; ++c) {
        double f2[5] = {0}, dg[15] = {0};
        for (int f = 0; f < 4; ++f) {
            int64_t fi = m->csr_face[c * 4 + f];
            double sg = m->csr_sign[c * 4 + f];
            for (int q = 0; q < 5; ++q) f2[q] += sg * rec2[fi * 20 + q];
            for (int q = 0; q < 15; ++q) dg[q] += sg * rec2[fi * 20 + 5 + q];
        }
        for (int q = 0; q < 5; ++q) W[q * nc + c] -= (S[c * 5 + q] + f2[q]) / m->vol[c];
        for (int q = 0; q < 15; ++q) dW[q * nc + c] = (G[c * 15 + q] + dg[q]) / m->vol[c];
    }
    free(rec1); free(rec2); free(Ws); free(dWs); free(S); free(G);
    return 0;
}
