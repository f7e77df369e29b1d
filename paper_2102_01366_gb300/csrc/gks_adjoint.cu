// gks_adjoint.cu -- reverse (adjoint) sweep of one two-stage step, FP64.
//
// Given the adjoint of the step's result, (lambda W^{n+1}, lambda grad
// W^{n+1}), these kernels return the adjoint of its start, (lambda W^n,
// lambda grad W^n): the transpose of the step's Jacobian applied to a vector,
// with the time step frozen.  Every part of the step but the kinetic solution
// at a Gauss point is linear in the working state (the linear-weight
// reconstruction, the evaluation of R at the Gauss points, the face frame
// rotations, the stage records of Eqs. linear-system and s2o4, the update of
// averages and of gradients by Eq. gauss-formula); those are transposed by
// hand, each as a gather so that no two threads write one location.  The
// kinetic solution (Eq. 2nd-flux with Eq. new-equ-part) is differentiated in
// reverse mode (gks_point_adj.cuh, about three point evaluations of work),
// inviscid or viscous.
//
//   k_adj_src2 / k_adj_src1  per-cell adjoints of the face-record sums
//   k_adj_point_rev<NR>      per (face, Gauss point): the point solution's
//                            adjoint in reverse mode
//   k_adj_face_back          per face: rotations and evaluation at the
//                            points transposed -> adjoints of both cells'
//                            reconstruction coefficients
//   k_adj_gather_poly        per cell: sum over its four faces
//   k_adj_recon_local        per cell: transpose of a = M2 d and of the
//                            monomial constant (linear weights)
//   k_adj_recon_weno         the same with the nonlinear WENO weights, and
//   k_adj_slopes             the neighbours' P1 slopes those weights use
//   k_adj_recon_gather       per cell: adjoint of its working state from its
//                            own and its neighbours' stencil adjoints
//   k_adj_final              the three paths into (W^n, grad W^n)
#include <cuda_runtime.h>

#include "gks_cells.cuh"
#include "gks_device.cuh"
#include "gks_face.cuh"
#include "gks_kernels.h"
#include "gks_point_adj.cuh"

namespace gks {

constexpr int ADJ_IN = 40;       // inputs of the point solution: WL, gL, WR, gR (face frame)
constexpr int ADJ_THREADS = 64;  // threads per block of k_adj_point_rev

// stage 2 records: [sum w 4/3 D (5) | sum w dW n (15)]; the cell sums enter
// W^{n+1} = W^n - (S + sum s rec[0:5]) / |Omega| and
// grad W^{n+1} = (G + sum s rec[5:20]) / |Omega|
__global__ void k_adj_src2(DevMesh<double> m, const double* __restrict__ lW, const double* __restrict__ ldW,
                           double* __restrict__ src) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m.nc) return;
    const double iv = m.inv_vol[c];
    double* o = src + c * 20;
    for (int q = 0; q < 5; ++q) o[q] = -lW[q * m.nc + c] * iv;
    for (int j = 0; j < 15; ++j) o[5 + j] = ldW[j * m.nc + c] * iv;
}

// stage 1 records: [sum w Fh | sum w (2 Fh - D/3) | sum w W* n | sum w W0 n];
// they enter W* = W^n - sum s rec[0:5] / |Omega|, S = sum s rec[5:10] (into
// W^{n+1} with -1/|Omega|), grad W* = sum s rec[10:25] / |Omega| and
// G = sum s rec[25:40] (into grad W^{n+1} with 1/|Omega|)
__global__ void k_adj_src1(DevMesh<double> m, const double* __restrict__ lW, const double* __restrict__ ldW,
                           const double* __restrict__ lXs, double* __restrict__ src) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m.nc) return;
    const double iv = m.inv_vol[c];
    const double* xs = lXs + c * XS;
    double* o = src + c * 40;
    for (int q = 0; q < 5; ++q) {
        o[q] = -xs[q] * iv;
        o[5 + q] = -lW[q * m.nc + c] * iv;
    }
    for (int j = 0; j < 15; ++j) {
        o[10 + j] = xs[5 + j] * iv;
        o[25 + j] = ldW[j * m.nc + c] * iv;
    }
}

// adjoint of eval_poly: lc += (d val / d c)^T lv + (d g / d c)^T lg
__device__ __forceinline__ void eval_poly_adj(const double* X, const double* lv, const double (*lg)[5],
                                              double* lc) {
    const double x = X[0], y = X[1], z = X[2];
    for (int q = 0; q < 5; ++q) {
        double* c = lc + q * 10;
        const double v = lv[q], g0 = lg[0][q], g1 = lg[1][q], g2 = lg[2][q];
        c[0] += v;
        c[1] += v * x + g0;
        c[2] += v * y + g1;
        c[3] += v * z + g2;
        c[4] += v * x * x + 2.0 * x * g0;
        c[5] += v * x * y + y * g0 + x * g1;
        c[6] += v * x * z + z * g0 + x * g2;
        c[7] += v * y * y + 2.0 * y * g1;
        c[8] += v * y * z + z * g1 + y * g2;
        c[9] += v * z * z + 2.0 * z * g2;
    }
}

// adjoint of to_local: (lW, lg) global from (lWt, lgt) in the face frame
__device__ __forceinline__ void to_local_adj(const double (*Rm)[3], const double* lWt, const double (*lgt)[5],
                                             double* lW, double (*lg)[5]) {
    lW[0] = lWt[0];
    lW[4] = lWt[4];
    for (int i = 0; i < 3; ++i) lW[1 + i] = Rm[0][i] * lWt[1] + Rm[1][i] * lWt[2] + Rm[2][i] * lWt[3];
    double lh[3][5];
    for (int j = 0; j < 3; ++j) {
        lh[j][0] = lgt[j][0];
        lh[j][4] = lgt[j][4];
        for (int l = 0; l < 3; ++l)
            lh[j][1 + l] = Rm[0][l] * lgt[j][1] + Rm[1][l] * lgt[j][2] + Rm[2][l] * lgt[j][3];
    }
    for (int i = 0; i < 3; ++i)
        for (int q = 0; q < 5; ++q) lg[i][q] = Rm[0][i] * lh[0][q] + Rm[1][i] * lh[1][q] + Rm[2][i] * lh[2][q];
}

// the momentum block of a global vector in the face frame (the adjoint of
// to_global)
__device__ __forceinline__ void rotate_in(const double (*Rm)[3], double* v) {
    const double a = v[1], b = v[2], c = v[3];
    for (int j = 0; j < 3; ++j) v[1 + j] = Rm[j][0] * a + Rm[j][1] * b + Rm[j][2] * c;
}

// The point's inputs in the face frame (WL, gL, WR, gR: 40 values) from the
// stored reconstruction, and the output adjoints of the point (face frame)
// from the record adjoints (the transposed record formulas of the stage).
template <int NR>
__device__ __forceinline__ void adj_point_setup(const DevMesh<double>& m, const double* __restrict__ poly,
                                                const double* __restrict__ Xavg, const double* __restrict__ src,
                                                int64_t f, int k, double (*Rm)[3], double* x, double* lFh,
                                                double* lD, double* lW0, double* ldWt,
                                                const Phys<double>* ph = nullptr) {
    const int L = m.flr[f], R = m.flr[m.nf + f];
    const double* geo = m.fgeo + f * FGEO;
    const double n[3] = {geo[0], geo[1], geo[2]};
    const double w = geo[3];
    face_frame(n, Rm);
    // record adjoints: the left cell adds the record, the right one subtracts it
    // (a boundary face has one cell)
    double lr[NR];
    for (int j = 0; j < NR; ++j)
        lr[j] = (L >= 0 ? src[(int64_t)L * NR + j] : 0.0) - (R >= 0 ? src[(int64_t)R * NR + j] : 0.0);
    for (int q = 0; q < 5; ++q) {
        double sn0 = 0.0, sn1 = 0.0;
        if (NR == 40) {
            for (int i = 0; i < 3; ++i) {
                sn0 += n[i] * lr[10 + 3 * q + i];
                sn1 += n[i] * lr[25 + 3 * q + i];
            }
            lFh[q] = w * (lr[q] + 2.0 * lr[5 + q]);
            lD[q] = -w * (1.0 / 3.0) * lr[5 + q];
            lW0[q] = w * (sn0 + sn1);
            ldWt[q] = 0.5 * w * sn0;
        } else {
            for (int i = 0; i < 3; ++i) sn0 += n[i] * lr[5 + 3 * q + i];
            lFh[q] = 0.0;
            lD[q] = w * (4.0 / 3.0) * lr[q];
            lW0[q] = 0.0;
            ldWt[q] = w * sn0;
        }
    }
    rotate_in(Rm, lFh);
    rotate_in(Rm, lD);
    rotate_in(Rm, lW0);
    rotate_in(Rm, ldWt);
    if (x) {
        // each side's state in the face frame, as the forward flux forms it
        for (int side = 0; side < 2; ++side) {
            const int cell = side == 0 ? L : R;
            const int in = side == 0 ? R : L;
            double* xs = x + 20 * side;
            double (*gs)[5] = reinterpret_cast<double (*)[5]>(xs + 5);
            double Wv[5], g[3][5];
            if (cell == FLR_OPEN) {
                // open: the interior cell's average, zero gradient
                for (int q = 0; q < 5; ++q) {
                    Wv[q] = Xavg[(int64_t)in * XS + q];
                    g[0][q] = g[1][q] = g[2][q] = 0.0;
                }
                to_local(Rm, Wv, g, xs, gs);
                continue;
            }
            if (cell == FLR_FIXED) {
                // fixed: the interior cell's fixed state carried to the point
                const int si = 1 - side;
                const double X[3] = {geo[4 + 9 * si + 3 * k], geo[5 + 9 * si + 3 * k], geo[6 + 9 * si + 3 * k]};
                fixed_ghost(m.fixed + (int64_t)in * XS, X, Wv, g);
                to_local(Rm, Wv, g, xs, gs);
                continue;
            }
            // a real side, or a wall side from the interior cell at the point
            const int src_side = cell >= 0 ? side : 1 - side;
            const int64_t c = cell >= 0 ? cell : in;
            const double X[3] = {geo[4 + 9 * src_side + 3 * k], geo[5 + 9 * src_side + 3 * k],
                                 geo[6 + 9 * src_side + 3 * k]};
            eval_poly(poly + c * POLY_STRIDE, X, Wv, g);
            to_local(Rm, Wv, g, xs, gs);
            if (cell == FLR_SLIP_WALL) slip_wall_ghost(xs, gs);
            if (cell == FLR_NOSLIP_WALL) noslip_wall_ghost(xs, gs);
            if (cell == FLR_ISOTHERMAL_WALL) isothermal_wall_ghost(xs, gs, ph->gm1, ph->twall);
            if (cell == FLR_MOVING_WALL) {
                double Uw[3];
                rotate_vec(Rm, ph->uwall, Uw);
                moving_wall_ghost(xs, gs, ph->gm1, Uw);
            }
        }
    }
}

// A forward-mode number (value and one derivative) for the Jacobian of the
// isothermal-wall ghost, the one nonlinear ghost.
struct Fwd {
    double v, d;
    __device__ Fwd() : v(0.0), d(0.0) {}
    __device__ Fwd(double x) : v(x), d(0.0) {}
    __device__ Fwd(double x, double dx) : v(x), d(dx) {}
};
__device__ __forceinline__ Fwd operator+(Fwd a, Fwd b) { return Fwd(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Fwd operator-(Fwd a, Fwd b) { return Fwd(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Fwd operator-(Fwd a) { return Fwd(-a.v, -a.d); }
__device__ __forceinline__ Fwd operator*(Fwd a, Fwd b) { return Fwd(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ Fwd operator/(Fwd a, Fwd b) {
    const double q = a.v / b.v;
    return Fwd(q, (a.d - q * b.d) / b.v);
}
__device__ __forceinline__ Fwd& operator+=(Fwd& a, Fwd b) { return a = a + b; }

// li += J^T ls for a nonlinear wall ghost G (isothermal or moving wall) at
// the interior face-frame state x (W, grad W: 20 values), by one forward pass
// per input; Uw is the wall velocity in the face frame
__device__ void wall_ghost_adj(int kind, const double* x, const double* ls, double gm1, double twall,
                               const double* Uw, double* li) {
    const Fwd Uwd[3] = {Fwd(Uw[0]), Fwd(Uw[1]), Fwd(Uw[2])};
    for (int i = 0; i < 20; ++i) {
        Fwd Wd[5], gd[3][5];
        for (int q = 0; q < 5; ++q) Wd[q] = Fwd(x[q], i == q ? 1.0 : 0.0);
        for (int j = 0; j < 3; ++j)
            for (int q = 0; q < 5; ++q) gd[j][q] = Fwd(x[5 + 5 * j + q], i == 5 + 5 * j + q ? 1.0 : 0.0);
        if (kind == FLR_ISOTHERMAL_WALL)
            isothermal_wall_ghost(Wd, gd, Fwd(gm1), Fwd(twall));
        else
            moving_wall_ghost(Wd, gd, Fwd(gm1), Uwd);
        double acc = 0.0;
        for (int q = 0; q < 5; ++q) acc += ls[q] * Wd[q].d;
        for (int j = 0; j < 3; ++j)
            for (int q = 0; q < 5; ++q) acc += ls[5 + 5 * j + q] * gd[j][q].d;
        li[i] += acc;
    }
}

// One thread per (face, Gauss point) of interior faces: the point
// solution's adjoint in reverse mode (gks_point_adj), lx[f][k][0:40].
template <int NR, bool VISC>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_point_rev(DevMesh<double> m, Phys<double> ph,
                                                               const double* __restrict__ poly,
                                                               const double* __restrict__ Xavg,
                                                               const double* __restrict__ src, double dt,
                                                               double* __restrict__ lx) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m.nf * 3) return;
    const int64_t f = t / 3;
    const int k = (int)(t - f * 3);
    double Rm[3][3], x[ADJ_IN], lFh[5], lD[5], lW0[5], ldWt[5];
    adj_point_setup<NR>(m, poly, Xavg, src, f, k, Rm, x, lFh, lD, lW0, ldWt, &ph);
    double* l = lx + t * ADJ_IN;
    double lin[ADJ_IN];
    for (int i = 0; i < ADJ_IN; ++i) lin[i] = 0.0;
    gks_point_adj<VISC>(ph, x, reinterpret_cast<const double (*)[5]>(x + 5), x + 20,
                  reinterpret_cast<const double (*)[5]>(x + 25), dt, lFh, lD, lW0, ldWt, lin,
                  reinterpret_cast<double (*)[5]>(lin + 5), lin + 20, reinterpret_cast<double (*)[5]>(lin + 25));
    for (int i = 0; i < ADJ_IN; ++i) l[i] = lin[i];
}

// One thread per face: the input adjoints of its three points carried back
// through the rotations and the evaluation at the points into
// lpf[f][side][5][10].
// A wall side's adjoint joins the interior side's at the same point (a
// mirror is its own transpose; the isothermal and moving walls' ghost
// Jacobians are transposed at the interior state); an open side's goes to the interior cell's average,
// lwo[f][5] (zero on every other face).
// XW: the mesh has isothermal or moving wall faces, whose ghosts' Jacobians
// (and the local frame they need) only those instances carry
template <bool XW>
__global__ void k_adj_face_back(DevMesh<double> m, const double* __restrict__ lx, double* __restrict__ lpf,
                                double* __restrict__ lwo, const double* __restrict__ poly, Phys<double> ph) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= m.nf) return;
    const int L = m.flr[f], R = m.flr[m.nf + f];
    const double* geo = m.fgeo + f * FGEO;
    const double n[3] = {geo[0], geo[1], geo[2]};
    double Rm[3][3];
    face_frame(n, Rm);
    double lp[2][50], lw[5] = {0, 0, 0, 0, 0};
    for (int j = 0; j < 50; ++j) lp[0][j] = lp[1][j] = 0.0;
    for (int k = 0; k < 3; ++k) {
        double l[ADJ_IN];
        for (int i = 0; i < ADJ_IN; ++i) l[i] = lx[(f * 3 + k) * ADJ_IN + i];
        for (int side = 0; side < 2; ++side) {
            const int cell = side == 0 ? L : R;
            if (cell >= 0) continue;
            double* ls = l + 20 * side;
            double (*lg)[5] = reinterpret_cast<double (*)[5]>(ls + 5);
            double* li = l + 20 * (1 - side);
            if (cell == FLR_OPEN) {
                double lW[5], lgg[3][5];
                to_local_adj(Rm, ls, lg, lW, lgg);
                for (int q = 0; q < 5; ++q) lw[q] += lW[q];
            } else if (cell == FLR_FIXED) {
                // a set fixed state is a constant of the step: nothing flows back
            } else if (XW && (cell == FLR_ISOTHERMAL_WALL || cell == FLR_MOVING_WALL)) {
                // the interior state at the point, face frame, then the ghost's transpose
                const int src_side = 1 - side;
                const int64_t c = side == 0 ? R : L;
                const double X[3] = {geo[4 + 9 * src_side + 3 * k], geo[5 + 9 * src_side + 3 * k],
                                     geo[6 + 9 * src_side + 3 * k]};
                double Wv[5], g[3][5], x[20];
                eval_poly(poly + c * POLY_STRIDE, X, Wv, g);
                to_local(Rm, Wv, g, x, reinterpret_cast<double (*)[5]>(x + 5));
                double Uw[3];
                rotate_vec(Rm, ph.uwall, Uw);
                wall_ghost_adj(cell, x, ls, ph.gm1, ph.twall, Uw, li);
            } else {
                if (cell == FLR_SLIP_WALL) slip_wall_ghost(ls, lg);
                if (cell == FLR_NOSLIP_WALL) noslip_wall_ghost(ls, lg);
                for (int i = 0; i < 20; ++i) li[i] += ls[i];
            }
        }
        for (int side = 0; side < 2; ++side) {
            if ((side == 0 ? L : R) < 0) continue;
            const double X[3] = {geo[4 + 9 * side + 3 * k], geo[5 + 9 * side + 3 * k], geo[6 + 9 * side + 3 * k]};
            double lW[5], lg[3][5];
            to_local_adj(Rm, l + 20 * side, reinterpret_cast<const double (*)[5]>(l + 20 * side + 5), lW, lg);
            eval_poly_adj(X, lW, lg, lp[side]);
        }
    }
    double* o = lpf + f * 100;
    for (int j = 0; j < 50; ++j) {
        o[j] = lp[0][j];
        o[50 + j] = lp[1][j];
    }
    for (int q = 0; q < 5; ++q) lwo[f * 5 + q] = lw[q];
}

// adjoint of a cell's reconstruction coefficients: the sum over its faces
__global__ void k_adj_gather_poly(DevMesh<double> m, const double* __restrict__ lpf, double* __restrict__ lp) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m.nc) return;
    double acc[50];
    for (int j = 0; j < 50; ++j) acc[j] = 0.0;
    for (int f = 0; f < 4; ++f) {
        const int e = m.cface[f * m.nc + c];
        const double* src = lpf + (int64_t)(e >> 1) * 100 + (e & 1) * 50;
        for (int j = 0; j < 50; ++j) acc[j] += src[j];
    }
    for (int j = 0; j < 50; ++j) lp[c * 50 + j] = acc[j];
}

// A cell whose reconstruction fell back to its average (the positivity
// check, Sec. 4.3: R = P0, zero slopes) passes only the adjoint of its
// constant on to its own average; nothing reaches the stencil data or the
// neighbours' slopes.  The fallback decision itself is piecewise constant.
__device__ __forceinline__ void fallback_back(const double* __restrict__ lp, int64_t c, int q,
                                              double* __restrict__ ld, double* __restrict__ lbn,
                                              double* __restrict__ own) {
    double* o = ld + (c * 5 + q) * 16;
    for (int j = 0; j < 16; ++j) o[j] = 0.0;
    if (lbn)
        for (int j = 0; j < 12; ++j) lbn[(c * 5 + q) * 12 + j] = 0.0;
    own[c * 5 + q] = lp[c * 50 + q * 10];
}

// Transpose of the linear-weight reconstruction of one cell (Sec. 4.1):
// R = a = M2 d, c0 = Q0 - sum_k R_k M_k (second moments), with
// d = [Q_nb - Q0 (4); grad Q_nb (12)].  Writes ld[c][q][16] = M2^T lambda_a
// and own[c][q] = lambda_c0 - sum over existing neighbours of ld[c][q][f].
__global__ void k_adj_recon_local(DevMesh<double> m, const double* __restrict__ lp, const int32_t* __restrict__ fb,
                                  double* __restrict__ ld, double* __restrict__ own) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m.nc * 5) return;
    const int64_t c = idx / 5;
    const int q = (int)(idx - c * 5);
    if (fb[c]) {
        fallback_back(lp, c, q, ld, nullptr, own);
        return;
    }
    const double* tile = m.tile + (c / CELLS_PER_BLOCK) * TILE_ROWS * CELLS_PER_BLOCK + c % CELLS_PER_BLOCK;
    auto T_ = [&](int row) { return tile[(int64_t)row * CELLS_PER_BLOCK]; };
    const double* l = lp + c * 50 + q * 10;
    const double lc0 = l[0];
    double la[9];
    for (int k = 0; k < 9; ++k) la[k] = l[1 + k];
    for (int k = 3; k < 9; ++k) la[k] -= lc0 * T_(TILE_MOM + (k - 3));
    double* o = ld + (c * 5 + q) * 16;
    double s = 0.0;
    for (int j = 0; j < 16; ++j) {
        double acc = 0.0;
        for (int k = 0; k < 9; ++k) acc += T_(TILE_M2 + k * 16 + j) * la[k];
        o[j] = acc;
    }
    for (int f = 0; f < 4; ++f)
        if (m.nbr[f * m.nc + c] >= 0) s += o[f];
    own[c * 5 + q] = lc0 - s;
}

// P1 slope of cell x for component q from the working state X (the
// reconstruction's step 1, Sec. 4.3)
__device__ __forceinline__ void adj_p1_slope(const DevMesh<double>& m, const double* __restrict__ X, int64_t x,
                                             int q, double* b) {
    const int64_t nc = m.nc;
    const double Qx = X[x * XS + q];
    b[0] = b[1] = b[2] = 0.0;
    for (int f = 0; f < 4; ++f) {
        const int nb = m.nbr[f * nc + x];
        if (nb < 0) continue;
        const double dq = X[(int64_t)nb * XS + q] - Qx;
        for (int i = 0; i < 3; ++i) b[i] += m.M1[(i * 4 + f) * nc + x] * dq;
    }
}

__device__ __forceinline__ double sgn(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0); }

// beta_0 of the two-step reconstruction (Eq. p0-non-linear-weight): the
// neighbours' P1 slopes b_j, beta_0j = |Omega|^{2/3} |b_j|^2, weights
// w1j = 1 + s1 / (eps + beta_0j) with s1 the 4/3 power of the mean pairwise
// |beta_0j - beta_0k|, beta_0 = sum w1j beta_0j / sum w1j; kept for the reverse.
struct Beta0 {
    double bj[4][3], b0j[4], w1j[4];
    double s1, ws, accb, sum, beta;
    int slot[4], nn, npair;
};

__device__ __forceinline__ void beta0_forward(const DevMesh<double>& m, const double* __restrict__ X,
                                              const int* nb, int q, double v23, double eps, Beta0& B) {
    B.nn = 0;
    for (int f = 0; f < 4; ++f) {
        if (nb[f] < 0) continue;
        adj_p1_slope(m, X, nb[f], q, B.bj[B.nn]);
        const double* bj = B.bj[B.nn];
        B.b0j[B.nn] = v23 * (bj[0] * bj[0] + bj[1] * bj[1] + bj[2] * bj[2]);
        B.slot[B.nn++] = f;
    }
    B.beta = B.s1 = B.ws = B.accb = B.sum = 0.0;
    B.npair = 0;
    if (B.nn > 0) {
        for (int j = 0; j < B.nn; ++j)
            for (int k = 0; k < j; ++k) {
                B.sum += fabs(B.b0j[j] - B.b0j[k]);
                ++B.npair;
            }
        B.s1 = B.npair ? pow43(B.sum / B.npair) : 0.0;
        for (int j = 0; j < B.nn; ++j) {
            B.w1j[j] = 1.0 + B.s1 / (eps + B.b0j[j]);
            B.ws += B.w1j[j];
            B.accb += B.w1j[j] * B.b0j[j];
        }
        B.beta = B.accb / B.ws;
    }
}

// adjoint of beta_0 into the adjoints of the neighbours' slopes lbj[j][3]
__device__ __forceinline__ void beta0_backward(const Beta0& B, double lbeta0, double v23, double eps,
                                               double (*lbj)[3]) {
    for (int j = 0; j < 4; ++j) lbj[j][0] = lbj[j][1] = lbj[j][2] = 0.0;
    if (B.nn == 0) return;
    const double lacc = lbeta0 / B.ws, lws = -lbeta0 * B.accb / (B.ws * B.ws);
    double lb0[4], ls1 = 0.0;
    for (int j = 0; j < B.nn; ++j) {
        const double lwj = lacc * B.b0j[j] + lws;
        lb0[j] = lacc * B.w1j[j] - lwj * B.s1 / ((eps + B.b0j[j]) * (eps + B.b0j[j]));
        ls1 += lwj / (eps + B.b0j[j]);
    }
    if (B.npair) {
        const double lsum = ls1 * (4.0 / 3.0) * cbrt(B.sum / B.npair) / B.npair;
        for (int j = 0; j < B.nn; ++j)
            for (int k = 0; k < B.nn; ++k)
                if (k != j) lb0[j] += lsum * sgn(B.b0j[j] - B.b0j[k]);
    }
    for (int j = 0; j < B.nn; ++j)
        for (int i = 0; i < 3; ++i) lbj[j][i] = 2.0 * v23 * B.bj[j][i] * lb0[j];
}

// the neighbours' slope adjoints into lbn[f][3] (zero for missing neighbours)
__device__ __forceinline__ void store_lbn(const Beta0& B, const double (*lbj)[3], double* __restrict__ ob) {
    for (int j = 0; j < 12; ++j) ob[j] = 0.0;
    for (int j = 0; j < B.nn; ++j)
        for (int i = 0; i < 3; ++i) ob[3 * B.slot[j] + i] = lbj[j][i];
}

// Transpose of the third-order multi-resolution WENO reconstruction of one
// cell and component (Sec. 4.2, 4.3): R = c2 a + cb b with the nonlinear
// weights of beta_0 (two-step, from the neighbours' P1 slopes), beta_1, beta_2;
// c0 = Q0 - sum_k R_k M_k.  The weights are recomputed from the stage's
// working state X and differentiated (|x|' = sign x, (x^{4/3})' = 4/3 x^{1/3}).
// Writes ld[c][q][16] (adjoint of the stencil data d), lbn[c][q][f][3] (of
// the neighbours' slopes as this cell uses them) and own[c][q] (of Q0 through
// c0 and the differences d[0:4]).
__global__ void k_adj_recon_weno(DevMesh<double> m, double eps, const double* __restrict__ X,
                                 const double* __restrict__ lp, const int32_t* __restrict__ fb,
                                 double* __restrict__ ld, double* __restrict__ lbn, double* __restrict__ own) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m.nc * 5) return;
    const int64_t c = idx / 5, nc = m.nc;
    const int q = (int)(idx - c * 5);
    if (fb[c]) {
        fallback_back(lp, c, q, ld, lbn, own);
        return;
    }
    const double* tile = m.tile + (c / CELLS_PER_BLOCK) * TILE_ROWS * CELLS_PER_BLOCK + c % CELLS_PER_BLOCK;
    auto T_ = [&](int row) { return tile[(int64_t)row * CELLS_PER_BLOCK]; };
    int nb[4];
    for (int f = 0; f < 4; ++f) nb[f] = m.nbr[f * nc + c];
    const double Q0 = X[c * XS + q];
    double d[16];
    for (int f = 0; f < 4; ++f) {
        const bool ok = nb[f] >= 0;
        const double* xn = X + (ok ? (int64_t)nb[f] : c) * XS;
        d[f] = ok ? xn[q] - Q0 : 0.0;
        for (int l = 0; l < 3; ++l) d[4 + 3 * f + l] = ok ? xn[5 + 3 * q + l] : 0.0;
    }
    double a[9];
    for (int k = 0; k < 9; ++k) {
        double acc = 0.0;
        for (int j = 0; j < 16; ++j) acc += T_(TILE_M2 + k * 16 + j) * d[j];
        a[k] = acc;
    }
    double Mm[6];
    for (int k = 0; k < 6; ++k) Mm[k] = T_(TILE_MOM + k);
    double b[3] = {0.0, 0.0, 0.0};
    for (int f = 0; f < 4; ++f) {
        if (nb[f] < 0) continue;
        for (int i = 0; i < 3; ++i) b[i] += T_(TILE_M1 + i * 4 + f) * d[f];
    }
    const double v23 = T_(TILE_V23), v43 = T_(TILE_V43);
    const double g22 = 100.0 / 111.0, g12 = 10.0 / 111.0, g02 = 1.0 / 111.0, g11 = 10.0 / 11.0;
    // forward: beta_1, beta_0 (two-step), beta_2, sigma, weights
    const double beta1 = v23 * (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    Beta0 B0;
    beta0_forward(m, X, nb, q, v23, eps, B0);
    const double beta0 = B0.beta;
    const double H[3][3] = {{2.0 * a[3], a[4], a[5]}, {a[4], 2.0 * a[6], a[7]}, {a[5], a[7], 2.0 * a[8]}};
    const double MM[3][3] = {{Mm[0], Mm[1], Mm[2]}, {Mm[1], Mm[3], Mm[4]}, {Mm[2], Mm[4], Mm[5]}};
    double first = 0.0, MH[3][3];
    for (int l = 0; l < 3; ++l) {
        for (int i = 0; i < 3; ++i) MH[l][i] = MM[i][0] * H[l][0] + MM[i][1] * H[l][1] + MM[i][2] * H[l][2];
        first += a[l] * a[l] + H[l][0] * MH[l][0] + H[l][1] * MH[l][1] + H[l][2] * MH[l][2];
    }
    const double second = H[0][0] * H[0][0] + a[4] * a[4] + a[5] * a[5] + H[1][1] * H[1][1] + a[7] * a[7] +
                          H[2][2] * H[2][2];
    const double beta2 = v23 * first + v43 * second;
    const double z = 0.5 * (fabs(beta2 - beta1) + fabs(beta2 - beta0));
    const double sigma = pow43(z);
    const double bet[3] = {beta0, beta1, beta2}, gam[3] = {g02, g12, g22};
    double r[3], w[3];
    for (int k = 0; k < 3; ++k) {
        r[k] = sigma / (eps + bet[k]);
        w[k] = gam[k] * (1.0 + r[k] * r[k]);
    }
    const double iw = 1.0 / (w[0] + w[1] + w[2]);
    const double c2 = (w[2] * iw) / g22;
    const double cb = (w[1] * iw) / g11 - c2 * g12 / g11;

    // reverse
    const double* l = lp + c * 50 + q * 10;
    const double lc0 = l[0];
    double lR[9];
    for (int k = 0; k < 9; ++k) lR[k] = l[1 + k];
    for (int k = 3; k < 9; ++k) lR[k] -= lc0 * Mm[k - 3];
    double la[9], lb[3], lc2 = 0.0, lcb = 0.0;
    for (int k = 0; k < 9; ++k) {
        la[k] = c2 * lR[k];
        lc2 += lR[k] * a[k];
    }
    for (int i = 0; i < 3; ++i) {
        lb[i] = cb * lR[i];
        lcb += lR[i] * b[i];
    }
    // c2 = w2 iw / g22, cb = w1 iw / g11 - c2 g12 / g11
    const double lc2t = lc2 - lcb * g12 / g11;
    double lw[3] = {0.0, lcb * iw / g11, lc2t * iw / g22};
    const double liw = lc2t * w[2] / g22 + lcb * w[1] / g11;
    const double lS = -liw * iw * iw;
    double lbet[3] = {0.0, 0.0, 0.0}, lsig = 0.0;
    for (int k = 0; k < 3; ++k) {
        lw[k] += lS;
        const double lr = lw[k] * gam[k] * 2.0 * r[k];
        lsig += lr / (eps + bet[k]);
        lbet[k] += -lr * sigma / ((eps + bet[k]) * (eps + bet[k]));
    }
    // sigma = z^{4/3}, z = (|b2 - b1| + |b2 - b0|) / 2
    const double lz = lsig * (4.0 / 3.0) * cbrt(z);
    const double s21 = sgn(beta2 - beta1), s20 = sgn(beta2 - beta0);
    lbet[2] += 0.5 * lz * (s21 + s20);
    lbet[1] += -0.5 * lz * s21;
    lbet[0] += -0.5 * lz * s20;
    // beta_2 = v23 first + v43 second
    const double lfirst = v23 * lbet[2], lsecond = v43 * lbet[2];
    double lH[3][3];
    for (int l2 = 0; l2 < 3; ++l2) {
        la[l2] += 2.0 * a[l2] * lfirst;
        for (int i = 0; i < 3; ++i) lH[l2][i] = 2.0 * MH[l2][i] * lfirst;
    }
    lH[0][0] += 2.0 * H[0][0] * lsecond;
    lH[1][1] += 2.0 * H[1][1] * lsecond;
    lH[2][2] += 2.0 * H[2][2] * lsecond;
    la[4] += 2.0 * a[4] * lsecond;
    la[5] += 2.0 * a[5] * lsecond;
    la[7] += 2.0 * a[7] * lsecond;
    la[3] += 2.0 * lH[0][0];
    la[4] += lH[0][1] + lH[1][0];
    la[5] += lH[0][2] + lH[2][0];
    la[6] += 2.0 * lH[1][1];
    la[7] += lH[1][2] + lH[2][1];
    la[8] += 2.0 * lH[2][2];
    // beta_1 = v23 |b|^2
    for (int i = 0; i < 3; ++i) lb[i] += 2.0 * v23 * b[i] * lbet[1];
    double lbj[4][3];
    beta0_backward(B0, lbet[0], v23, eps, lbj);
    // a = M2 d, b = M1 d[0:4]
    double* o = ld + (c * 5 + q) * 16;
    double s = 0.0;
    for (int j = 0; j < 16; ++j) {
        double acc = 0.0;
        for (int k = 0; k < 9; ++k) acc += T_(TILE_M2 + k * 16 + j) * la[k];
        if (j < 4 && nb[j] >= 0)
            for (int i = 0; i < 3; ++i) acc += T_(TILE_M1 + i * 4 + j) * lb[i];
        o[j] = acc;
        if (j < 4 && nb[j] >= 0) s += acc;
    }
    own[c * 5 + q] = lc0 - s;
    store_lbn(B0, lbj, lbn + (c * 5 + q) * 12);
}

// Transpose of the second-order WENO reconstruction R^2nd (Eq.
// final_weno_expression-2nd) of one cell and component: R = Q0 + cb b.x with
// cb = (w1 / (w0 + w1)) / g11, w0, w1 from beta_0 (two-step) and beta_1,
// sigma = |beta_1 - beta_0|^{4/3}.  Same outputs as k_adj_recon_weno.
__global__ void k_adj_recon_weno2(DevMesh<double> m, double eps, const double* __restrict__ X,
                                  const double* __restrict__ lp, const int32_t* __restrict__ fb,
                                  double* __restrict__ ld, double* __restrict__ lbn, double* __restrict__ own) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m.nc * 5) return;
    const int64_t c = idx / 5, nc = m.nc;
    const int q = (int)(idx - c * 5);
    if (fb[c]) {
        fallback_back(lp, c, q, ld, lbn, own);
        return;
    }
    const double* tile = m.tile + (c / CELLS_PER_BLOCK) * TILE_ROWS * CELLS_PER_BLOCK + c % CELLS_PER_BLOCK;
    auto T_ = [&](int row) { return tile[(int64_t)row * CELLS_PER_BLOCK]; };
    int nb[4];
    for (int f = 0; f < 4; ++f) nb[f] = m.nbr[f * nc + c];
    const double Q0 = X[c * XS + q];
    double d[4];
    for (int f = 0; f < 4; ++f) d[f] = nb[f] >= 0 ? X[(int64_t)nb[f] * XS + q] - Q0 : 0.0;
    double b[3] = {0.0, 0.0, 0.0};
    for (int f = 0; f < 4; ++f) {
        if (nb[f] < 0) continue;
        for (int i = 0; i < 3; ++i) b[i] += T_(TILE_M1 + i * 4 + f) * d[f];
    }
    const double v23 = T_(TILE_V23);
    const double g01 = 1.0 / 11.0, g11 = 10.0 / 11.0;
    const double beta1 = v23 * (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    Beta0 B0;
    beta0_forward(m, X, nb, q, v23, eps, B0);
    const double beta0 = B0.beta;
    const double z = fabs(beta1 - beta0);
    const double sigma = pow43(z);
    const double bet[2] = {beta0, beta1}, gam[2] = {g01, g11};
    double r[2], w[2];
    for (int k = 0; k < 2; ++k) {
        r[k] = sigma / (eps + bet[k]);
        w[k] = gam[k] * (1.0 + r[k] * r[k]);
    }
    const double wsum = w[0] + w[1];
    const double cb = w[1] / (wsum * g11);

    // reverse: only the constant and the linear coefficients of R are nonzero
    const double* l = lp + c * 50 + q * 10;
    const double lc0 = l[0];
    double lb[3], lcb = 0.0;
    for (int i = 0; i < 3; ++i) {
        lb[i] = cb * l[1 + i];
        lcb += l[1 + i] * b[i];
    }
    double lw[2];
    const double lwsum = -lcb * w[1] / (wsum * wsum * g11);
    lw[0] = lwsum;
    lw[1] = lwsum + lcb / (wsum * g11);
    double lbet[2] = {0.0, 0.0}, lsig = 0.0;
    for (int k = 0; k < 2; ++k) {
        const double lr = lw[k] * gam[k] * 2.0 * r[k];
        lsig += lr / (eps + bet[k]);
        lbet[k] += -lr * sigma / ((eps + bet[k]) * (eps + bet[k]));
    }
    const double lz = lsig * (4.0 / 3.0) * cbrt(z);
    const double s10 = sgn(beta1 - beta0);
    lbet[1] += lz * s10;
    lbet[0] -= lz * s10;
    for (int i = 0; i < 3; ++i) lb[i] += 2.0 * v23 * b[i] * lbet[1];
    double lbj[4][3];
    beta0_backward(B0, lbet[0], v23, eps, lbj);
    double* o = ld + (c * 5 + q) * 16;
    double s = 0.0;
    for (int j = 0; j < 16; ++j) o[j] = 0.0;
    for (int j = 0; j < 4; ++j) {
        if (nb[j] < 0) continue;
        for (int i = 0; i < 3; ++i) o[j] += T_(TILE_M1 + i * 4 + j) * lb[i];
        s += o[j];
    }
    own[c * 5 + q] = lc0 - s;
    store_lbn(B0, lbj, lbn + (c * 5 + q) * 12);
}

// Transpose of the second-order reconstruction with linear weights: R = P1,
// the step-1 slope b = M1 d[0:4].
__global__ void k_adj_recon_p1(DevMesh<double> m, const double* __restrict__ lp, const int32_t* __restrict__ fb,
                               double* __restrict__ ld, double* __restrict__ own) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m.nc * 5) return;
    const int64_t c = idx / 5;
    const int q = (int)(idx - c * 5);
    if (fb[c]) {
        fallback_back(lp, c, q, ld, nullptr, own);
        return;
    }
    const double* tile = m.tile + (c / CELLS_PER_BLOCK) * TILE_ROWS * CELLS_PER_BLOCK + c % CELLS_PER_BLOCK;
    const double* l = lp + c * 50 + q * 10;
    double* o = ld + (c * 5 + q) * 16;
    double s = 0.0;
    for (int j = 0; j < 16; ++j) o[j] = 0.0;
    for (int j = 0; j < 4; ++j) {
        if (m.nbr[j * m.nc + c] < 0) continue;
        for (int i = 0; i < 3; ++i) o[j] += tile[(int64_t)(TILE_M1 + i * 4 + j) * CELLS_PER_BLOCK] * l[1 + i];
        s += o[j];
    }
    own[c * 5 + q] = l[0] - s;
}

// Adjoint of the neighbours' P1 slopes, per cell n and component: the slope
// adjoints the cells around n hold for n's slope (lbn, in the slot that
// points back to n) are summed, then carried through n's slope operator:
// lds[n][q][f] is the adjoint of Q_nbr(n, f) - Q_n.
__global__ void k_adj_slopes(DevMesh<double> m, const int8_t* __restrict__ rev, const double* __restrict__ lbn,
                             double* __restrict__ lds) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m.nc * 5) return;
    const int64_t n = idx / 5, nc = m.nc;
    const int q = (int)(idx - n * 5);
    double ls[3] = {0.0, 0.0, 0.0};
    for (int f = 0; f < 4; ++f) {
        const int c = m.nbr[f * nc + n];
        if (c < 0) continue;
        const double* src = lbn + ((int64_t)c * 5 + q) * 12 + 3 * rev[f * nc + n];
        for (int i = 0; i < 3; ++i) ls[i] += src[i];
    }
    double* o = lds + (n * 5 + q) * 4;
    for (int f = 0; f < 4; ++f)
        o[f] = m.nbr[f * nc + n] >= 0
                   ? m.M1[(0 * 4 + f) * nc + n] * ls[0] + m.M1[(1 * 4 + f) * nc + n] * ls[1] +
                         m.M1[(2 * 4 + f) * nc + n] * ls[2]
                   : 0.0;
}

// adjoint of a cell's working state [W (5), grad W (15)]: its own part and,
// from each neighbour n, the entries of n's stencil adjoint in the slot that
// points back to this cell across the shared face (rev[f][c])
__global__ void k_adj_recon_gather(DevMesh<double> m, const int8_t* __restrict__ rev,
                                   const double* __restrict__ ld, const double* __restrict__ lds,
                                   const double* __restrict__ own, const double* __restrict__ lwo,
                                   double* __restrict__ lX) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m.nc * 5) return;
    const int64_t c = idx / 5;
    const int q = (int)(idx - c * 5);
    double lq = own[c * 5 + q];
    // open faces of this cell: their ghost is this cell's average
    for (int f = 0; f < 4; ++f) {
        const int e = m.cface[f * m.nc + c];
        const int64_t face = e >> 1;
        if (m.flr[(int64_t)(1 - (e & 1)) * m.nf + face] == FLR_OPEN) lq += lwo[face * 5 + q];
    }
    double lg[3] = {0.0, 0.0, 0.0};
    for (int f = 0; f < 4; ++f) {
        const int n = m.nbr[f * m.nc + c];
        if (n < 0) continue;
        const int r = rev[f * m.nc + c];
        const double* o = ld + ((int64_t)n * 5 + q) * 16;
        lq += o[r];
        for (int l = 0; l < 3; ++l) lg[l] += o[4 + 3 * r + l];
        if (lds) lq += lds[((int64_t)n * 5 + q) * 4 + r] - lds[(c * 5 + q) * 4 + f];
    }
    double* x = lX + c * XS;
    x[q] = lq;
    for (int l = 0; l < 3; ++l) x[5 + 3 * q + l] = lg[l];
}

// lambda W^n = lambda W^{n+1} (the update's pass-through) + lambda W* (the
// stage-1 pass-through) + the stage-1 reconstruction's; lambda grad W^n from
// the stage-1 reconstruction alone
__global__ void k_adj_final(DevMesh<double> m, const double* __restrict__ lW, const double* __restrict__ lXs,
                            const double* __restrict__ lX1, double* __restrict__ oW, double* __restrict__ odW) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m.nc) return;
    for (int q = 0; q < 5; ++q) oW[q * m.nc + c] = lW[q * m.nc + c] + lXs[c * XS + q] + lX1[c * XS + q];
    for (int j = 0; j < 15; ++j) odW[j * m.nc + c] = lX1[c * XS + 5 + j];
}

// --------------------------------------------------------------------------
// launcher
// --------------------------------------------------------------------------
static inline unsigned grid_of(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

static Phys<double> phys64(const HostPhys& p) {
    Phys<double> ph;
    ph.gamma = p.gamma;
    ph.gm1 = p.gamma - 1.0;
    ph.K = (5.0 - 3.0 * p.gamma) / (p.gamma - 1.0);
    ph.tau_eps = p.tau_eps;
    ph.tau_c = p.tau_c;
    ph.mu = p.mu;
    ph.eps_w = p.eps_weno;
    ph.viscous = p.viscous;
    ph.smooth = p.smooth;
    ph.prf = p.prf;
    ph.twall = p.twall;
    for (int i = 0; i < 3; ++i) ph.uwall[i] = p.uwall[i];
    return ph;
}

// transpose of one stage's reconstruction: lp (per-cell coefficient
// adjoints) into lX, from the stage's working state X
static void recon_back(const DevMesh<double>& m, const HostPhys& p, const AdjBuffers& b, const double* X,
                       const int32_t* fb,
                       double* lX, cudaStream_t s) {
    const int B = 128;
    if (p.weno) {
        if (p.order == 2)
            k_adj_recon_weno2<<<grid_of(m.nc * 5, B), B, 0, s>>>(m, p.eps_weno, X, b.lp, fb, b.ld, b.lbn, b.own);
        else
            k_adj_recon_weno<<<grid_of(m.nc * 5, B), B, 0, s>>>(m, p.eps_weno, X, b.lp, fb, b.ld, b.lbn, b.own);
        k_adj_slopes<<<grid_of(m.nc * 5, B), B, 0, s>>>(m, b.rev, b.lbn, b.lds);
        k_adj_recon_gather<<<grid_of(m.nc * 5, B), B, 0, s>>>(m, b.rev, b.ld, b.lds, b.own, b.lwo, lX);
    } else {
        if (p.order == 2)
            k_adj_recon_p1<<<grid_of(m.nc * 5, B), B, 0, s>>>(m, b.lp, fb, b.ld, b.own);
        else
            k_adj_recon_local<<<grid_of(m.nc * 5, B), B, 0, s>>>(m, b.lp, fb, b.ld, b.own);
        k_adj_recon_gather<<<grid_of(m.nc * 5, B), B, 0, s>>>(m, b.rev, b.ld, nullptr, b.own, b.lwo, lX);
    }
}

// transpose of one stage's face flux: the record adjoints in b.src into the
// per-cell reconstruction-coefficient adjoints b.lp
template <int NR>
static void flux_back(const DevMesh<double>& m, const Phys<double>& ph, const AdjBuffers& b, const double* poly,
                      const double* X, double dt, cudaStream_t s) {
    const int B = 128;
    if (ph.viscous)
        k_adj_point_rev<NR, true><<<grid_of(m.nf * 3, ADJ_THREADS), ADJ_THREADS, 0, s>>>(m, ph, poly, X, b.src, dt,
                                                                                       b.lx);
    else
        k_adj_point_rev<NR, false><<<grid_of(m.nf * 3, ADJ_THREADS), ADJ_THREADS, 0, s>>>(m, ph, poly, X, b.src, dt,
                                                                                        b.lx);
    if (m.xwalls)
        k_adj_face_back<true><<<grid_of(m.nf, B), B, 0, s>>>(m, b.lx, b.lpf, b.lwo, poly, ph);
    else
        k_adj_face_back<false><<<grid_of(m.nf, B), B, 0, s>>>(m, b.lx, b.lpf, b.lwo, poly, ph);
    k_adj_gather_poly<<<grid_of(m.nc, B), B, 0, s>>>(m, b.lpf, b.lp);
}

// The reverse sweep proper; the forward intermediates (the two stages'
// working states X1, X2 and reconstructions poly1, poly2) come from a forward
// recomputation by the caller.
cudaError_t adjoint_reverse(const DevMesh<double>& m, const HostPhys& p, double dt, const AdjBuffers& b,
                            const double* X1, const double* X2, const double* lW, const double* ldW, double* oW,
                            double* odW, cudaStream_t s) {
    const Phys<double> ph = phys64(p);
    const int B = 128;
    cudaError_t e;
    // stage 2
    k_adj_src2<<<grid_of(m.nc, B), B, 0, s>>>(m, lW, ldW, b.src);
    flux_back<20>(m, ph, b, b.poly2, X2, dt, s);
    recon_back(m, p, b, X2, b.fallback + m.nc, b.lXs, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // stage 1
    k_adj_src1<<<grid_of(m.nc, B), B, 0, s>>>(m, lW, ldW, b.lXs, b.src);
    flux_back<40>(m, ph, b, b.poly1, X1, dt, s);
    recon_back(m, p, b, X1, b.fallback, b.lX1, s);
    k_adj_final<<<grid_of(m.nc, B), B, 0, s>>>(m, lW, b.lXs, b.lX1, oW, odW);
    return cudaGetLastError();
}

}  // namespace gks
