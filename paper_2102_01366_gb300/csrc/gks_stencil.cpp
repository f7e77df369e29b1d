// gks_stencil.cpp -- FP64 least-squares operators of the compact
// reconstruction (Sec. 4.1 and Sec. 4.3), built once per mesh on the host.
//
// P1 (Eq. p1-stenci-condition): slopes b from the neighbours' averages in the
// least-squares sense, M1 = R^-1 Q^T from a Householder QR of the offsets.
//
// P2 (Eqs. large-stenci-condition-1/2): P2 = Qbar_0 + sum_k a_k p^k with the
// zero-mean basis of Eq. base (x, y, z, xx, xy, xz, yy, yz, zz about the
// centroid).  The neighbours' averages are matched exactly, the neighbours'
// averaged gradients in the least-squares sense.  Solved by the null-space
// method: a QR of the constraint matrix splits a into a constrained part
// and a free part, and the free part is the least-squares solution of the
// projected gradient rows (a second QR).  Unknowns are scaled by powers of
// h0 = |Omega|^(1/3) and gradient rows by h0 so that both QRs work on O(1)
// entries; the result is unscaled before it is stored.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>

#include "gks_internal.h"

namespace gks {
namespace {

// Householder QR of A (m x n, m >= n, row-major).  On return Q (m x m) and
// R (n x n, upper) satisfy A = Q[:, :n] R.
void householder_qr(int m, int n, const double* A, double* Q, double* R) {
    double W[16 * 16];
    std::memcpy(W, A, sizeof(double) * m * n);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) Q[i * m + j] = i == j ? 1.0 : 0.0;
    double v[16];
    for (int k = 0; k < n; ++k) {
        double norm = 0.0;
        for (int i = k; i < m; ++i) norm += W[i * n + k] * W[i * n + k];
        norm = std::sqrt(norm);
        if (norm == 0.0) continue;
        double alpha = W[k * n + k] > 0.0 ? -norm : norm;
        for (int i = 0; i < m; ++i) v[i] = 0.0;
        for (int i = k; i < m; ++i) v[i] = W[i * n + k];
        v[k] -= alpha;
        double vn = 0.0;
        for (int i = k; i < m; ++i) vn += v[i] * v[i];
        if (vn == 0.0) continue;
        // W <- (I - 2 v v^T / vn) W
        for (int j = k; j < n; ++j) {
            double s = 0.0;
            for (int i = k; i < m; ++i) s += v[i] * W[i * n + j];
            s *= 2.0 / vn;
            for (int i = k; i < m; ++i) W[i * n + j] -= s * v[i];
        }
        // Q <- Q (I - 2 v v^T / vn)
        for (int i = 0; i < m; ++i) {
            double s = 0.0;
            for (int l = k; l < m; ++l) s += Q[i * m + l] * v[l];
            s *= 2.0 / vn;
            for (int l = k; l < m; ++l) Q[i * m + l] -= s * v[l];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) R[i * n + j] = j >= i ? W[i * n + j] : 0.0;
}

// condition proxy: smallest over largest |R_ii|
double diag_ratio(int n, const double* R) {
    double lo = INFINITY, hi = 0.0;
    for (int i = 0; i < n; ++i) {
        double d = std::fabs(R[i * n + i]);
        lo = std::fmin(lo, d);
        hi = std::fmax(hi, d);
    }
    return hi > 0.0 ? lo / hi : 0.0;
}

// X (n x r) <- R^-1 X for upper-triangular R (n x n)
void upper_solve(int n, const double* R, int r, double* X) {
    for (int c = 0; c < r; ++c)
        for (int i = n - 1; i >= 0; --i) {
            double s = X[i * r + c];
            for (int j = i + 1; j < n; ++j) s -= R[i * n + j] * X[j * r + c];
            X[i * r + c] = s / R[i * n + i];
        }
}

// X (n x r) <- R^-T X for upper-triangular R (n x n)
void lower_solve_transposed(int n, const double* R, int r, double* X) {
    for (int c = 0; c < r; ++c)
        for (int i = 0; i < n; ++i) {
            double s = X[i * r + c];
            for (int j = 0; j < i; ++j) s -= R[j * n + i] * X[j * r + c];
            X[i * r + c] = s / R[i * n + i];
        }
}

const int PI_[6] = {0, 0, 0, 1, 1, 2};
const int PJ_[6] = {0, 1, 2, 1, 2, 2};

bool cell_stencil(const gks_mesh& m, int64_t c, double* M1, double* M2) {
    int fl[4], nn = 0;
    double d[4][3];
    for (int f = 0; f < 4; ++f) {
        int64_t nb = m.nbr[c * 4 + f];
        if (nb < 0) continue;
        for (int a = 0; a < 3; ++a)
            d[nn][a] = (m.cen[nb * 3 + a] + (double)m.nbr_img[(c * 4 + f) * 3 + a] * m.per(c)[a]) -
                       m.cen[c * 3 + a];
        fl[nn++] = f;
    }
    std::memset(M1, 0, sizeof(double) * 12);
    std::memset(M2, 0, sizeof(double) * 144);
    if (nn < 3) return false;
    const double h0 = std::cbrt(m.vol[c]);

    // ---- P1: min |A b - dq|, A rows d_f / h0 ----------------------------
    {
        double A[4 * 3], Q[16], R[9];
        for (int r = 0; r < nn; ++r)
            for (int a = 0; a < 3; ++a) A[r * 3 + a] = d[r][a] / h0;
        householder_qr(nn, 3, A, Q, R);
        if (diag_ratio(3, R) < 1e-12) return false;
        double X[3 * 4];
        for (int i = 0; i < 3; ++i)
            for (int r = 0; r < nn; ++r) X[i * nn + r] = Q[r * nn + i];  // Q1^T
        upper_solve(3, R, nn, X);
        for (int i = 0; i < 3; ++i)
            for (int r = 0; r < nn; ++r) M1[i * 4 + fl[r]] = X[i * nn + r] / h0;
    }

    // ---- P2: constrained least squares ----------------------------------
    double sc[9];
    for (int k = 0; k < 9; ++k) sc[k] = k < 3 ? h0 : h0 * h0;
    const double* M0 = &m.mom2[c * 6];
    double C[4 * 9];        // constraint rows (neighbour averages of the basis)
    double B[12 * 9];       // gradient rows
    const int nb_rows = 3 * nn;
    for (int r = 0; r < nn; ++r) {
        int64_t nb = m.nbr[c * 4 + fl[r]];
        const double* Mn = &m.mom2[nb * 6];
        for (int k = 0; k < 3; ++k) C[r * 9 + k] = d[r][k] / sc[k];
        for (int q = 0; q < 6; ++q)
            C[r * 9 + 3 + q] = (Mn[q] - M0[q] + d[r][PI_[q]] * d[r][PJ_[q]]) / sc[3 + q];
        for (int l = 0; l < 3; ++l) {
            double* row = &B[(3 * r + l) * 9];
            for (int k = 0; k < 3; ++k) row[k] = (k == l ? h0 : 0.0) / sc[k];
            for (int q = 0; q < 6; ++q) {
                double g = (PI_[q] == l ? d[r][PJ_[q]] : 0.0) + (PJ_[q] == l ? d[r][PI_[q]] : 0.0);
                row[3 + q] = h0 * g / sc[3 + q];
            }
        }
    }
    // QR of C^T (9 x nn)
    double Ct[9 * 4], Qc[81], Rc[16];
    for (int k = 0; k < 9; ++k)
        for (int r = 0; r < nn; ++r) Ct[k * nn + r] = C[r * 9 + k];
    householder_qr(9, nn, Ct, Qc, Rc);
    if (diag_ratio(nn, Rc) < 1e-12) return false;
    const int nz = 9 - nn;
    // BQ2 (nb_rows x nz), BQ1 (nb_rows x nn)
    double BQ2[12 * 6], BQ1[12 * 4];
    for (int i = 0; i < nb_rows; ++i) {
        for (int j = 0; j < nz; ++j) {
            double s = 0.0;
            for (int k = 0; k < 9; ++k) s += B[i * 9 + k] * Qc[k * 9 + nn + j];
            BQ2[i * nz + j] = s;
        }
        for (int j = 0; j < nn; ++j) {
            double s = 0.0;
            for (int k = 0; k < 9; ++k) s += B[i * 9 + k] * Qc[k * 9 + j];
            BQ1[i * nn + j] = s;
        }
    }
    double Qb[144], Rb[36];
    householder_qr(nb_rows, nz, BQ2, Qb, Rb);
    if (diag_ratio(nz, Rb) < 1e-12) return false;
    // Z = Q2 Rb^-1 Qb1^T  (9 x nb_rows)
    double Y[6 * 12];
    for (int j = 0; j < nz; ++j)
        for (int i = 0; i < nb_rows; ++i) Y[j * nb_rows + i] = Qb[i * nb_rows + j];
    upper_solve(nz, Rb, nb_rows, Y);
    double Z[9 * 12];
    for (int k = 0; k < 9; ++k)
        for (int i = 0; i < nb_rows; ++i) {
            double s = 0.0;
            for (int j = 0; j < nz; ++j) s += Qc[k * 9 + nn + j] * Y[j * nb_rows + i];
            Z[k * nb_rows + i] = s;
        }
    // X = Rc^-T (nn x nn) applied to the identity
    double X[16];
    for (int i = 0; i < nn; ++i)
        for (int j = 0; j < nn; ++j) X[i * nn + j] = i == j ? 1.0 : 0.0;
    lower_solve_transposed(nn, Rc, nn, X);
    // Mq = Q1 X - Z BQ1 X  (9 x nn)
    double BX[12 * 4];
    for (int i = 0; i < nb_rows; ++i)
        for (int j = 0; j < nn; ++j) {
            double s = 0.0;
            for (int l = 0; l < nn; ++l) s += BQ1[i * nn + l] * X[l * nn + j];
            BX[i * nn + j] = s;
        }
    for (int k = 0; k < 9; ++k) {
        for (int j = 0; j < nn; ++j) {
            double s = 0.0;
            for (int l = 0; l < nn; ++l) s += Qc[k * 9 + l] * X[l * nn + j];
            for (int i = 0; i < nb_rows; ++i) s -= Z[k * nb_rows + i] * BX[i * nn + j];
            M2[k * 16 + fl[j]] = s / sc[k];
        }
        for (int r = 0; r < nn; ++r)
            for (int l = 0; l < 3; ++l)
                M2[k * 16 + 4 + 3 * fl[r] + l] = Z[k * nb_rows + 3 * r + l] * h0 / sc[k];
    }
    return true;
}

}  // namespace

// Sec. 4.4, boundary cells of the linear-weight (smooth) reconstruction: a
// first-order polynomial fitted to the P2 stencil's data by least squares,
// the neighbours' averages (rows d_f . b = dQ_f) and averaged gradients
// (rows b = grad Q_f), each gradient row scaled by h0 = |Omega|^(1/3) as in
// the P2 system.  Written into the 9 x 16 layout of M2 (the quadratic rows
// zero); false when the cell has fewer than 3 neighbours or the fit is
// singular.
bool cell_linear_fit(const gks_mesh& m, int64_t c, double* M2) {
    int fl[4], nn = 0;
    double d[4][3];
    for (int f = 0; f < 4; ++f) {
        int64_t nb = m.nbr[c * 4 + f];
        if (nb < 0) continue;
        for (int a = 0; a < 3; ++a)
            d[nn][a] = (m.cen[nb * 3 + a] + (double)m.nbr_img[(c * 4 + f) * 3 + a] * m.per(c)[a]) -
                       m.cen[c * 3 + a];
        fl[nn++] = f;
    }
    std::memset(M2, 0, sizeof(double) * 144);
    if (nn < 3) return false;
    const double h0 = std::cbrt(m.vol[c]);
    // unknown y = h0 b; rows: (d_f / h0) . y = dQ_f, then y_l = h0 dQ_f/dx_l
    const int rows = 4 * nn;
    double A[16 * 3], Q[256], R[9];
    for (int r = 0; r < nn; ++r)
        for (int a = 0; a < 3; ++a) A[r * 3 + a] = d[r][a] / h0;
    for (int r = 0; r < nn; ++r)
        for (int l = 0; l < 3; ++l)
            for (int a = 0; a < 3; ++a) A[(nn + 3 * r + l) * 3 + a] = a == l ? 1.0 : 0.0;
    householder_qr(rows, 3, A, Q, R);
    if (diag_ratio(3, R) < 1e-12) return false;
    double X[3 * 16];
    for (int i = 0; i < 3; ++i)
        for (int r = 0; r < rows; ++r) X[i * rows + r] = Q[r * rows + i];  // Q1^T
    upper_solve(3, R, rows, X);
    for (int k = 0; k < 3; ++k)
        for (int r = 0; r < nn; ++r) {
            M2[k * 16 + fl[r]] = X[k * rows + r] / h0;
            for (int l = 0; l < 3; ++l) M2[k * 16 + 4 + 3 * fl[r] + l] = X[k * rows + nn + 3 * r + l];
        }
    return true;
}

gks_status build_stencils(gks_mesh& m) {
    m.M1.assign((size_t)m.nc * 12, 0.0);
    m.M2.assign((size_t)m.nc * 144, 0.0);
    m.singular.assign((size_t)m.nc, 0);
    // independent per cell: split the cells over the host's hardware threads
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int64_t nthr = std::min<int64_t>((int64_t)hw, std::max<int64_t>(1, m.nc / 4096));
    auto work = [&](int64_t lo, int64_t hi) {
        for (int64_t c = lo; c < hi; ++c) {
            if (!cell_stencil(m, c, &m.M1[c * 12], &m.M2[c * 144])) {
                m.singular[c] = 1;
                std::memset(&m.M1[c * 12], 0, sizeof(double) * 12);
                std::memset(&m.M2[c * 144], 0, sizeof(double) * 144);
            }
        }
    };
    std::vector<std::thread> pool;
    const int64_t chunk = (m.nc + nthr - 1) / nthr;
    for (int64_t t = 1; t < nthr; ++t)
        pool.emplace_back(work, std::min(m.nc, t * chunk), std::min(m.nc, (t + 1) * chunk));
    work(0, std::min(m.nc, chunk));
    for (auto& th : pool) th.join();
    m.n_singular = 0;
    for (int64_t c = 0; c < m.nc; ++c) m.n_singular += m.singular[c];
    m.has_stencils = true;
    return GKS_OK;
}

}  // namespace gks

namespace gks {
namespace {

// Least squares with equality constraints by the null-space method: over x
// (n unknowns) minimise |A x - h| subject to E x = g, E (ne x n, full row
// rank), A (nl x n).  The solution is linear in (g, h): x = Pe g + Pl h,
// written to Pe (n x ne) and Pl (n x nl).  A QR of E^T splits x into the
// part fixed by the constraints, Q1 R^-T g, and a free part Q2 z; z is the
// least-squares solution of (A Q2) z = h - A Q1 R^-T g (a second QR).
// False when either factor is numerically singular.
bool constrained_ls(int n, int ne, const double* E, int nl, const double* A, double* Pe, double* Pl) {
    const int nz = n - ne;
    if (ne < 1 || nz < 0 || nl < nz) return false;
    double Et[9 * 9], Qe[81], Re[81];
    for (int i = 0; i < n; ++i)
        for (int r = 0; r < ne; ++r) Et[i * ne + r] = E[r * n + i];
    householder_qr(n, ne, Et, Qe, Re);
    if (diag_ratio(ne, Re) < 1e-12) return false;
    // G = R^-T (ne x ne): the constrained part is Q1 G g
    double G[81];
    for (int i = 0; i < ne; ++i)
        for (int j = 0; j < ne; ++j) G[i * ne + j] = i == j ? 1.0 : 0.0;
    lower_solve_transposed(ne, Re, ne, G);
    double Q1G[9 * 9];  // n x ne
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < ne; ++j) {
            double s = 0.0;
            for (int l = 0; l < ne; ++l) s += Qe[i * n + l] * G[l * ne + j];
            Q1G[i * ne + j] = s;
        }
    if (nz == 0) {
        std::memcpy(Pe, Q1G, sizeof(double) * n * ne);
        std::memset(Pl, 0, sizeof(double) * n * nl);
        return true;
    }
    // AQ2 (nl x nz), AQ1G (nl x ne)
    double AQ2[16 * 9], AQ1G[16 * 9];
    for (int r = 0; r < nl; ++r) {
        for (int j = 0; j < nz; ++j) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += A[r * n + k] * Qe[k * n + ne + j];
            AQ2[r * nz + j] = s;
        }
        for (int j = 0; j < ne; ++j) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += A[r * n + k] * Q1G[k * ne + j];
            AQ1G[r * ne + j] = s;
        }
    }
    double Qa[256], Ra[81];
    householder_qr(nl, nz, AQ2, Qa, Ra);
    if (diag_ratio(nz, Ra) < 1e-12) return false;
    // Z = Ra^-1 Qa1^T (nz x nl): z = Z (h - AQ1G g)
    double Z[9 * 16];
    for (int j = 0; j < nz; ++j)
        for (int r = 0; r < nl; ++r) Z[j * nl + r] = Qa[r * nl + j];
    upper_solve(nz, Ra, nl, Z);
    for (int i = 0; i < n; ++i) {
        for (int r = 0; r < nl; ++r) {
            double s = 0.0;
            for (int j = 0; j < nz; ++j) s += Qe[i * n + ne + j] * Z[j * nl + r];
            Pl[i * nl + r] = s;
        }
        for (int c = 0; c < ne; ++c) {
            double s = Q1G[i * ne + c];
            for (int r = 0; r < nl; ++r) s -= Pl[i * nl + r] * AQ1G[r * ne + c];
            Pe[i * ne + c] = s;
        }
    }
    return true;
}

}  // namespace

bool has_wall_face(const gks_mesh& m, int64_t c) {
    for (int f = 0; f < 4; ++f)
        if (m.nbr[c * 4 + f] < 0 && m.bkind[m.csr_face[c * 4 + f]] == GKS_BC_NOSLIP_WALL) return true;
    return false;
}

// Sec. 4.4: a cell with non-slip adiabatic wall faces reconstructs its
// momenta by constrained least squares, the wall velocity (zero) imposed on
// the polynomial at the wall faces -- at each face's centroid for the step-1
// P1, at its three Gauss points for the step-2 P2 (the unconstrained P2's
// data, with the wall rows as further equality constraints).  The imposed
// value is zero, so the result is linear in the stencil data and the cell
// average Q0:
//   W1 [3][5]:  b = W1 [dQ_f (4); Q0]
//   W2 [9][17]: a = W2 [dQ_f (4); grad Q_f (12); Q0]   (zero-mean basis)
// Used when there are at least 3 neighbours + wall faces, at most 3 wall
// faces, at most 9 equality rows in step 2 (neighbours + 3 per wall face)
// and at least 9 rows in all.
bool cell_wall_stencil(const gks_mesh& m, int64_t c, double* W2, double* W1) {
    int fl[4], wl[4], nn = 0, nw = 0;
    double d[4][3];
    for (int f = 0; f < 4; ++f) {
        int64_t nb = m.nbr[c * 4 + f];
        if (nb >= 0) {
            for (int a = 0; a < 3; ++a)
                d[nn][a] = (m.cen[nb * 3 + a] + (double)m.nbr_img[(c * 4 + f) * 3 + a] * m.per(c)[a]) -
                           m.cen[c * 3 + a];
            fl[nn++] = f;
        } else if (m.bkind[m.csr_face[c * 4 + f]] == GKS_BC_NOSLIP_WALL) {
            wl[nw++] = f;
        }
    }
    std::memset(W1, 0, sizeof(double) * 15);
    std::memset(W2, 0, sizeof(double) * 153);
    if (nw == 0 || nn + nw < 3 || nw > 3 || nn + 3 * nw > 9 || 4 * nn + 3 * nw < 9) return false;
    const double h0 = std::cbrt(m.vol[c]);
    // each wall face's Gauss points relative to the cell centroid
    double xg[4][3][3];
    for (int w = 0; w < nw; ++w) {
        const int64_t fi = m.csr_face[c * 4 + wl[w]];
        const double* gp = m.csr_sign[c * 4 + wl[w]] > 0 ? &m.gp_l[fi * 9] : &m.gp_r[fi * 9];
        for (int g = 0; g < 3; ++g)
            for (int a = 0; a < 3; ++a) xg[w][g][a] = gp[g * 3 + a];
    }
    // ---- step 1: unknown y = h0 b; rows scaled by 1 / h0 ------------------
    {
        double E[3 * 3], A[4 * 3], Pe[3 * 3], Pl[3 * 4];
        for (int w = 0; w < nw; ++w)
            for (int a = 0; a < 3; ++a)
                E[w * 3 + a] = (xg[w][0][a] + xg[w][1][a] + xg[w][2][a]) / (3.0 * h0);  // the face centroid
        for (int r = 0; r < nn; ++r)
            for (int a = 0; a < 3; ++a) A[r * 3 + a] = d[r][a] / h0;
        if (!constrained_ls(3, nw, E, nn, A, Pe, Pl)) return false;
        for (int i = 0; i < 3; ++i) {
            for (int r = 0; r < nn; ++r) W1[i * 5 + fl[r]] = Pl[i * nn + r] / h0;
            double q0 = 0.0;  // each wall row asks for b . x_w = -Q0
            for (int w = 0; w < nw; ++w) q0 -= Pe[i * nw + w];
            W1[i * 5 + 4] = q0 / h0;
        }
    }
    // ---- step 2: unknowns scaled by powers of h0 as the unconstrained P2 ---
    double sc[9];
    for (int k = 0; k < 9; ++k) sc[k] = k < 3 ? h0 : h0 * h0;
    const double* M0 = &m.mom2[c * 6];
    const int ne = nn + 3 * nw, nl = 3 * nn;
    double E[9 * 9], A[12 * 9], Pe[9 * 9], Pl[9 * 12];
    for (int r = 0; r < nn; ++r) {
        const double* Mn = &m.mom2[m.nbr[c * 4 + fl[r]] * 6];
        for (int k = 0; k < 3; ++k) E[r * 9 + k] = d[r][k] / sc[k];
        for (int q = 0; q < 6; ++q)
            E[r * 9 + 3 + q] = (Mn[q] - M0[q] + d[r][PI_[q]] * d[r][PJ_[q]]) / sc[3 + q];
        for (int l = 0; l < 3; ++l) {
            double* row = &A[(3 * r + l) * 9];
            for (int k = 0; k < 3; ++k) row[k] = (k == l ? h0 : 0.0) / sc[k];
            for (int q = 0; q < 6; ++q) {
                double g = (PI_[q] == l ? d[r][PJ_[q]] : 0.0) + (PJ_[q] == l ? d[r][PI_[q]] : 0.0);
                row[3 + q] = h0 * g / sc[3 + q];
            }
        }
    }
    for (int w = 0; w < nw; ++w)
        for (int g = 0; g < 3; ++g) {
            double* row = &E[(nn + 3 * w + g) * 9];
            const double* X = xg[w][g];
            for (int k = 0; k < 3; ++k) row[k] = X[k] / sc[k];
            for (int q = 0; q < 6; ++q) row[3 + q] = (X[PI_[q]] * X[PJ_[q]] - M0[q]) / sc[3 + q];
        }
    if (!constrained_ls(9, ne, E, nl, A, Pe, Pl)) return false;
    for (int k = 0; k < 9; ++k) {
        for (int r = 0; r < nn; ++r) {
            W2[k * 17 + fl[r]] = Pe[k * ne + r] / sc[k];
            for (int l = 0; l < 3; ++l) W2[k * 17 + 4 + 3 * fl[r] + l] = Pl[k * nl + 3 * r + l] * h0 / sc[k];
        }
        double q0 = 0.0;  // each wall row asks for P2(x_g) - Q0 = -Q0
        for (int w = 0; w < 3 * nw; ++w) q0 -= Pe[k * ne + nn + w];
        W2[k * 17 + 16] = q0 / sc[k];
    }
    return true;
}

}  // namespace gks
