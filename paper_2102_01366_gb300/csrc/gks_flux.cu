// gks_flux.cu -- face flux kernels (Sec. 2.2, 3, 4.4, 4.5), sm_103a, FP64 and
// FP32-bulk instantiations.
//
//   k_flux         face-ordered, 6 threads per face (3 Gauss points x 2
//                  sides): R of both cells at the Gauss points, face frame,
//                  kinetic solution (Eq. 2nd-flux with the equilibrium state
//                  of Eq. new-equ-part), weighted face record of the stage
//                  (Sec. 3 Eqs. linear-system, s2o4, step-du); FP32
//   k_flux_single  the same with one thread per Gauss point; FP64
//
// Boundary faces take their ghost side from the face's kind (Sec. 4.4 slip
// wall, a fixed state, or zeroth-order extrapolation).
#include <cuda_runtime.h>

#include "gks_device.cuh"
#include "gks_face.cuh"
#include "gks_kernels.h"

namespace gks {

// --------------------------------------------------------------------------
// face flux
// --------------------------------------------------------------------------


// Face flux with 6 threads per face: 3 Gauss points x 2 sides.  The two sides
// of a Gauss point sit in different warps (warps 0-2 left, 3-5 right) so that
// no warp diverges on the side; the interface equilibrium, its slopes and the
// partial outputs are exchanged through shared memory:
//   phase 1  own side: state at the point, face frame, slopes, rho <psi>+-
//   phase 2  W^c, collision times; own kinetic part; rho <a_i psi>+-
//   phase 3  right warps form the equilibrium slopes (once per point) and
//            share a^c; then left warps add the C2 (a^c.u) flux terms,
//            right warps the C1, C3 flux terms and the dW term
//   phase 4  left warps finish the flux entries, right warps the gradient
//            entries of the record; the 3 points of each face are summed.
constexpr int FP_GP = 3 * FLUX_FACES;  // Gauss points per block (96)

template <typename T, int NR>
struct FluxSmem {
    T w0[2][FP_GP][5];   // rho <psi>+- of each side
    T p[2][FP_GP];       // pressure of each side
    T dwc[2][FP_GP][15]; // rho <a_i psi>+- of each side
    T ac[FP_GP][15];     // equilibrium slopes a^c_i (formed once, by the right warps)
    T out[2][FP_GP][20]; // partial Fh, D, W0, dW of each side
    T red[FP_GP * NR];   // weighted record entries per Gauss point
};

// The two warps that hold the two sides of the same 32 Gauss points (warp w
// and warp w + 3) exchange through shared memory only with each other, so
// they meet at a named barrier of their own instead of the whole block's.
__device__ __forceinline__ void pair_barrier(int g) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + (g >> 5)), "r"(64) : "memory");
}

template <typename T, int NR, int MINB, bool PRF>
__global__ void __launch_bounds__(2 * FP_GP, MINB) k_flux(DevMesh<T> m, Phys<T> ph,
                                                     const T* __restrict__ Wavg,
                                                     const T* __restrict__ poly,
                                                     T* __restrict__ rec,
                                                     const double* __restrict__ ctrl,
                                                     double dt_override) {
    __shared__ FluxSmem<T, NR> sm;
    const int side = threadIdx.x >= FP_GP ? 1 : 0;
    const int g = threadIdx.x - side * FP_GP;  // Gauss point within the block
    const int lf = g / 3;
    const int k = g - 3 * lf;
    const int64_t f0 = (int64_t)blockIdx.x * FLUX_FACES + lf;
    const bool active = f0 < m.nf;
    const int64_t f = active ? f0 : m.nf - 1;  // idle points compute a valid face, store nothing
    const int L = m.flr[f], Rc = m.flr[m.nf + f];
    // the face's case step; a finished case (dt = 0) computes with a dummy
    // step and its cells ignore the record
    const double dtc = ctrl ? ctrl[m.cell_case[L >= 0 ? L : Rc]] : dt_override;
    const T dt = dtc > 0.0 ? (T)dtc : T(1);
    const T* geo = m.fgeo + f * FGEO;
    const T n[3] = {geo[0], geo[1], geo[2]};
    const T w = geo[3];

    // ---- phase 1 ----
    const int mine = side == 0 ? L : Rc;
    const bool wall =
        mine == FLR_SLIP_WALL || mine == FLR_NOSLIP_WALL || mine == FLR_ISOTHERMAL_WALL || mine == FLR_MOVING_WALL;
    T Ws[5], gs[3][5];
    if (mine >= 0 || wall) {
        // a wall side starts from the interior cell's value at the point
        const int src = mine >= 0 ? side : 1 - side;
        const int64_t cell = mine >= 0 ? mine : (side == 0 ? Rc : L);
        const T X[3] = {geo[4 + 9 * src + 3 * k], geo[5 + 9 * src + 3 * k], geo[6 + 9 * src + 3 * k]};
        eval_poly(poly + cell * POLY_STRIDE, X, Ws, gs);
    } else if (mine == FLR_FIXED) {
        const int64_t in = side == 0 ? Rc : L;
        const int src = 1 - side;
        const T X[3] = {geo[4 + 9 * src + 3 * k], geo[5 + 9 * src + 3 * k], geo[6 + 9 * src + 3 * k]};
        fixed_ghost(m.fixed + in * XS, X, Ws, gs);
    } else {
        // open boundary: the missing side is the interior cell's average with
        // zero gradient (zeroth-order extrapolation; the paper leaves outflow
        // boundaries open, and copying the interior Gauss-point state is not
        // stable)
        const int64_t in = side == 0 ? Rc : L;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            Ws[q] = Wavg[in * XS + q];
            gs[0][q] = gs[1][q] = gs[2][q] = T(0);
        }
    }
    T Rm[3][3];
    face_frame(n, Rm);
    T tW[5], tg[3][5];
    to_local(Rm, Ws, gs, tW, tg);
    if (mine == FLR_SLIP_WALL) slip_wall_ghost(tW, tg);
    if (mine == FLR_NOSLIP_WALL) noslip_wall_ghost(tW, tg);
    if (mine == FLR_ISOTHERMAL_WALL) isothermal_wall_ghost(tW, tg, ph.gm1, ph.twall);
    if (mine == FLR_MOVING_WALL) {
        T Uw[3];
        rotate_vec(Rm, ph.uwall, Uw);
        moving_wall_ghost(tW, tg, ph.gm1, Uw);
    }
    const Prim<T> S = to_prim(tW, ph.gm1);
    Tab<T> t;
    T a[3][5], A[5];
    kinetic_side(ph, S, tg, side == 0 ? +1 : -1, t, a, A);
    T mw0[5] = {T(0), T(0), T(0), T(0), T(0)};
    acc_psi<0, 0, 0>(t, S.rho, mw0);
#pragma unroll
    for (int q = 0; q < 5; ++q) sm.w0[side][g][q] = mw0[q];
    sm.p[side][g] = S.p;
    pair_barrier(g);

    // ---- phase 2 ----
    T Wc[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) Wc[q] = sm.w0[0][g][q] + sm.w0[1][g][q];
    const Prim<T> C = to_prim(Wc, ph.gm1);
    const TimeCoef<T> tc = time_coefs(ph, sm.p[0][g], sm.p[1][g], C.p, dt);
    const T tau = tc.tau;
    T Fh[5], D[5], W0[5], dWt[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) Fh[q] = D[q] = W0[q] = dWt[q] = T(0);
    {
        T dwc[3][5];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
#pragma unroll
            for (int q = 0; q < 5; ++q) dwc[i][q] = T(0);
            acc_apsi<0, 0, 0>(t, a[i], S.rho, dwc[i]);
#pragma unroll
            for (int q = 0; q < 5; ++q) sm.dwc[side][g][5 * i + q] = dwc[i][q];
        }
    }
    if (!ph.smooth) {
        T mf0[5] = {0}, mf1[5] = {0}, mw1[5] = {0};
        acc_psi<1, 0, 0>(t, S.rho, mf0);
        acc_grad<1>(t, a, S.rho, mf1);
        acc_grad<0>(t, a, S.rho, mw1);
        axpy5(tc.k0, mf0, Fh);
        axpy5(-(tau * tc.k0 + tc.k1), mf1, Fh);
        axpy5(tc.dk0, mf0, D);
        axpy5(-(tau * tc.dk0 + tc.dk1), mf1, D);
        axpy5(T(1), mw0, W0);
        axpy5(-tau, mw1, W0);
        axpy5(tau - (tau + dt) * tc.E, mw1, dWt);
        T mw2[5] = {T(0), T(0), T(0), T(0), T(0)};
        if (ph.viscous) {
            T mf2[5] = {0};
            acc_apsi<1, 0, 0>(t, A, S.rho, mf2);
            acc_apsi<0, 0, 0>(t, A, S.rho, mw2);
            axpy5(-tau * tc.k0, mf2, Fh);
            axpy5(-tau * tc.dk0, mf2, D);
            axpy5(-tau, mw2, W0);
            axpy5(tau * (T(1) - tc.E), mw2, dWt);
        }
        if (PRF) {
            // this side's state integrals for the Pr fix, parked in its own
            // output slots until phase 3 ends
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                sm.out[side][g][q] = tc.k0 * mw0[q] - (tau * tc.k0 + tc.k1) * mw1[q] - tau * tc.k0 * mw2[q];
                sm.out[side][g][5 + q] =
                    tc.dk0 * mw0[q] - (tau * tc.dk0 + tc.dk1) * mw1[q] - tau * tc.dk0 * mw2[q];
            }
        }
    } else if (PRF) {
#pragma unroll
        for (int q = 0; q < 10; ++q) sm.out[side][g][q] = T(0);
    }
    pair_barrier(g);

    // ---- phase 3 ----
    {
        make_tab(t, C, ph.K, 0);
        T ac[3][5], Ac[5], rA[5];
        if (side == 1) {
            // the equilibrium slopes, once per point (Eq. co for g^c)
            T dWc[3][5];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int q = 0; q < 5; ++q) dWc[i][q] = sm.dwc[0][g][5 * i + q] + sm.dwc[1][g][5 * i + q];
            state_slopes(C, t, ph.K, dWc, ac, Ac, rA);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int q = 0; q < 5; ++q) sm.ac[g][5 * i + q] = ac[i][q];
        }
        pair_barrier(g);
        // Pr fix: the state integrals move to this side's (now unused) slope
        // slots; the right side adds the equilibrium part below
        T IW[10];
        if (PRF) {
#pragma unroll
            for (int q = 0; q < 10; ++q) IW[q] = sm.out[side][g][q];
        }
        if (side == 0) {
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int q = 0; q < 5; ++q) ac[i][q] = sm.ac[g][5 * i + q];
            T mf1[5] = {T(0), T(0), T(0), T(0), T(0)};
            acc_grad<1>(t, ac, C.rho, mf1);
            if (ph.smooth) {
                axpy5(-tau * T(0.5) * dt, mf1, Fh);
            } else {
                axpy5(tc.q2, mf1, Fh);
                axpy5(tc.dq2, mf1, D);
            }
        } else {
            T mf0[5] = {0}, mf2[5] = {0}, mw1[5];
            acc_psi<1, 0, 0>(t, C.rho, mf0);
            acc_apsi<1, 0, 0>(t, Ac, C.rho, mf2);
#pragma unroll
            for (int q = 0; q < 5; ++q) mw1[q] = -C.rho * rA[q];  // rho sum_i <(a_i . psi) u_i psi> (Eq. co)
            if (ph.smooth) {
                const T hd = T(0.5) * dt;
                axpy5(hd, mf0, Fh);
                axpy5(T(0.5) * hd * hd - tau * hd, mf2, Fh);
                axpy5(T(0.25) * dt * dt, mf2, D);
#pragma unroll
                for (int q = 0; q < 5; ++q) W0[q] = Wc[q];  // tau terms cancel: <(a.u + A) psi> = 0
                axpy5(-dt, mw1, dWt);
                if (PRF) {
#pragma unroll
                    for (int q = 0; q < 5; ++q) {
                        IW[q] += hd * Wc[q] - T(0.5) * hd * hd * mw1[q];
                        IW[5 + q] += -T(0.25) * dt * dt * mw1[q];
                    }
                }
            } else {
                axpy5(tc.q1, mf0, Fh);
                axpy5(tc.q3, mf2, Fh);
                axpy5(tc.dq1, mf0, D);
                axpy5(tc.dq3, mf2, D);
                const T C2 = (dt + tau) * tc.E - tau, C3 = dt - tau + tau * tc.E;
                axpy5(C2 - C3, mw1, dWt);
                if (PRF) {
#pragma unroll
                    for (int q = 0; q < 5; ++q) {
                        IW[q] += tc.q1 * Wc[q] + (tc.q2 - tc.q3) * mw1[q];
                        IW[5 + q] += tc.dq1 * Wc[q] + (tc.dq2 - tc.dq3) * mw1[q];
                    }
                }
            }
        }
        if (PRF) {
#pragma unroll
            for (int q = 0; q < 10; ++q) sm.dwc[side][g][q] = IW[q];
        }
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        sm.out[side][g][q] = Fh[q];
        sm.out[side][g][5 + q] = D[q];
        sm.out[side][g][10 + q] = W0[q];
        sm.out[side][g][15 + q] = dWt[q];
    }
    pair_barrier(g);

    // ---- phase 4: left warps the flux entries, right warps the gradient entries
    T* mine_rec = sm.red + g * NR;
    if (side == 0) {
        T Fs[5], Ds[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            Fs[q] = sm.out[0][g][q] + sm.out[1][g][q];
            Ds[q] = sm.out[0][g][5 + q] + sm.out[1][g][5 + q];
        }
        if (PRF) {
            T IWh[5], IWd[5], Wc[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                IWh[q] = sm.dwc[0][g][q] + sm.dwc[1][g][q];
                IWd[q] = sm.dwc[0][g][5 + q] + sm.dwc[1][g][5 + q];
                Wc[q] = sm.w0[0][g][q] + sm.w0[1][g][q];
            }
            const T U[3] = {Wc[1] / Wc[0], Wc[2] / Wc[0], Wc[3] / Wc[0]};
            prandtl_fix(ph.prf, U, IWh, Fs);
            prandtl_fix(ph.prf, U, IWd, Ds);
        }
        to_global(Rm, Fs);
        to_global(Rm, Ds);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            if (NR == 40) {
                // dt L + dt^2/6 L_t = 8/3 Fh - 1/3 F = 2 Fh - D / 3 (Eqs. linear-system, s2o4)
                mine_rec[q] = w * Fs[q];
                mine_rec[5 + q] = w * (T(2) * Fs[q] - Ds[q] * T(1.0 / 3.0));
            } else {
                mine_rec[q] = w * T(4.0 / 3.0) * Ds[q];  // dt^2/3 L_t(W*) = 4/3 (F* - 2 Fh*)
            }
        }
    } else {
        T Zs[5], Ys[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            Zs[q] = sm.out[0][g][10 + q] + sm.out[1][g][10 + q];
            Ys[q] = sm.out[0][g][15 + q] + sm.out[1][g][15 + q];
        }
        to_global(Rm, Zs);
        to_global(Rm, Ys);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            if (NR == 40) {
                const T ws = w * (Zs[q] + T(0.5) * Ys[q]);  // f* = f^n + dt/2 f_t^n
                const T w0 = w * Zs[q];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    mine_rec[10 + 3 * q + i] = ws * n[i];
                    mine_rec[25 + 3 * q + i] = w0 * n[i];
                }
            } else {
                const T dg = w * Ys[q];  // f^{n+1} = f^n + dt f_t^*
#pragma unroll
                for (int i = 0; i < 3; ++i) mine_rec[5 + 3 * q + i] = dg * n[i];
            }
        }
    }
    __syncthreads();
    // sum the three Gauss points of each face; coalesced record store
    const int64_t base = (int64_t)blockIdx.x * FLUX_FACES;
    for (int idx = threadIdx.x; idx < FLUX_FACES * NR; idx += 2 * FP_GP) {
        const int fl = idx / NR, j = idx - fl * NR;
        if (base + fl < m.nf) {
            const T* r = sm.red + fl * 3 * NR + j;
            rec[(base + fl) * NR + j] = (r[0] + r[NR]) + r[2 * NR];
        }
    }
}

// 3 threads per face, one Gauss point each (used for FP64, whose register
// footprint leaves no room for the lane-pair split)
template <typename T, int NR>
__global__ void __launch_bounds__(3 * FLUX_FACES) k_flux_single(DevMesh<T> m, Phys<T> ph,
                                                                 const T* __restrict__ Wavg,
                                                                 const T* __restrict__ poly,
                                                                 T* __restrict__ rec,
                                                                 const double* __restrict__ ctrl,
                                                                 double dt_override) {
    __shared__ T red[FLUX_FACES * 3 * NR];
    const int lf = threadIdx.x / 3;
    const int k = threadIdx.x - 3 * lf;
    const int64_t f = (int64_t)blockIdx.x * FLUX_FACES + lf;
    T* mine = red + (lf * 3 + k) * NR;
    if (f < m.nf) {
        const int L = m.flr[f], Rc = m.flr[m.nf + f];
        const double dtc = ctrl ? ctrl[m.cell_case[L >= 0 ? L : Rc]] : dt_override;
        const T dt = dtc > 0.0 ? (T)dtc : T(1);
        const T* geo = m.fgeo + f * FGEO;
        const T n[3] = {geo[0], geo[1], geo[2]};
        const T w = geo[3];
        T WL[5], gL[3][5], WR[5], gR[3][5];
        for (int side = 0; side < 2; ++side) {
            const int cell = side == 0 ? L : Rc;
            T* Wv = side == 0 ? WL : WR;
            T (*g)[5] = side == 0 ? gL : gR;
            if (cell >= 0 || cell == FLR_SLIP_WALL || cell == FLR_NOSLIP_WALL || cell == FLR_ISOTHERMAL_WALL ||
                cell == FLR_MOVING_WALL) {
                // a wall side starts from the interior cell's value at the point
                const int src = cell >= 0 ? side : 1 - side;
                const int64_t c = cell >= 0 ? cell : (side == 0 ? Rc : L);
                const T X[3] = {geo[4 + 9 * src + 3 * k], geo[5 + 9 * src + 3 * k], geo[6 + 9 * src + 3 * k]};
                eval_poly(poly + c * POLY_STRIDE, X, Wv, g);
            } else if (cell == FLR_FIXED) {
                const int64_t in = side == 0 ? Rc : L;
                const int src = 1 - side;
                const T X[3] = {geo[4 + 9 * src + 3 * k], geo[5 + 9 * src + 3 * k], geo[6 + 9 * src + 3 * k]};
                fixed_ghost(m.fixed + in * XS, X, Wv, g);
            } else {
                // open boundary: interior cell average, zero gradient
                const int64_t in = side == 0 ? Rc : L;
                for (int q = 0; q < 5; ++q) {
                    Wv[q] = Wavg[in * XS + q];
                    g[0][q] = g[1][q] = g[2][q] = T(0);
                }
            }
        }
        T Rm[3][3];
        face_frame(n, Rm);
        T tWL[5], tgL[3][5], tWR[5], tgR[3][5];
        to_local(Rm, WL, gL, tWL, tgL);
        to_local(Rm, WR, gR, tWR, tgR);
        if (L == FLR_SLIP_WALL) slip_wall_ghost(tWL, tgL);
        if (Rc == FLR_SLIP_WALL) slip_wall_ghost(tWR, tgR);
        if (L == FLR_NOSLIP_WALL) noslip_wall_ghost(tWL, tgL);
        if (Rc == FLR_NOSLIP_WALL) noslip_wall_ghost(tWR, tgR);
        if (L == FLR_ISOTHERMAL_WALL) isothermal_wall_ghost(tWL, tgL, ph.gm1, ph.twall);
        if (Rc == FLR_ISOTHERMAL_WALL) isothermal_wall_ghost(tWR, tgR, ph.gm1, ph.twall);
        if (L == FLR_MOVING_WALL || Rc == FLR_MOVING_WALL) {
            T Uw[3];
            rotate_vec(Rm, ph.uwall, Uw);
            if (L == FLR_MOVING_WALL) moving_wall_ghost(tWL, tgL, ph.gm1, Uw);
            if (Rc == FLR_MOVING_WALL) moving_wall_ghost(tWR, tgR, ph.gm1, Uw);
        }
        T Fh[5], D[5], W0[5], dWt[5];
        gks_point(ph, tWL, tgL, tWR, tgR, dt, Fh, D, W0, dWt);
        to_global(Rm, Fh);
        to_global(Rm, D);
        to_global(Rm, W0);
        to_global(Rm, dWt);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            if (NR == 40) {
                mine[q] = w * Fh[q];
                mine[5 + q] = w * (T(2) * Fh[q] - D[q] * T(1.0 / 3.0));
                const T ws = w * (W0[q] + T(0.5) * dWt[q]);
                const T w0 = w * W0[q];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    mine[10 + 3 * q + i] = ws * n[i];
                    mine[25 + 3 * q + i] = w0 * n[i];
                }
            } else {
                mine[q] = w * T(4.0 / 3.0) * D[q];
                const T dg = w * dWt[q];
#pragma unroll
                for (int i = 0; i < 3; ++i) mine[5 + 3 * q + i] = dg * n[i];
            }
        }
    }
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * FLUX_FACES;
    for (int idx = threadIdx.x; idx < FLUX_FACES * NR; idx += 3 * FLUX_FACES) {
        const int fl = idx / NR, j = idx - fl * NR;
        if (base + fl < m.nf) {
            const T* r = red + fl * 3 * NR + j;
            rec[(base + fl) * NR + j] = (r[0] + r[NR]) + r[2 * NR];
        }
    }
}

// --------------------------------------------------------------------------
// launcher
// --------------------------------------------------------------------------
template <typename T>
static Phys<T> make_phys(const HostPhys& p) {
    Phys<T> ph;
    ph.gamma = (T)p.gamma;
    ph.gm1 = (T)(p.gamma - 1.0);
    ph.K = (T)((5.0 - 3.0 * p.gamma) / (p.gamma - 1.0));
    ph.tau_eps = (T)p.tau_eps;
    ph.tau_c = (T)p.tau_c;
    ph.mu = (T)p.mu;
    ph.eps_w = (T)p.eps_weno;
    ph.viscous = p.viscous;
    ph.smooth = p.smooth;
    ph.prf = (T)p.prf;
    ph.twall = (T)p.twall;
    for (int i = 0; i < 3; ++i) ph.uwall[i] = (T)p.uwall[i];
    return ph;
}


template <typename T>
cudaError_t Launch<T>::flux(const DevMesh<T>& m, const HostPhys& p, const T* W, const T* poly, T* rec,
                            const double* ctrl, double dt_override, int stage, cudaStream_t s, int variant) {
    // ctrl is the per-case step array (NULL: dt_override everywhere)
    if (m.nf == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((m.nf + FLUX_FACES - 1) / FLUX_FACES);
    const Phys<T> ph = make_phys<T>(p);
    if constexpr (sizeof(T) == 4) {
        // FP32: the two sides of each Gauss point in separate warps; variant
        // 1 trades registers for occupancy (3 blocks per SM), variant 0 keeps
        // 2 blocks per SM without spills; the Pr fix has its own instances
        const bool prf = p.prf != 0.0;
        auto go = [&](auto kernel) { kernel<<<grid, 2 * FP_GP, 0, s>>>(m, ph, W, poly, rec, ctrl, dt_override); };
        if (variant == 1) {
            if (stage == 1)
                prf ? go(k_flux<T, 40, 3, true>) : go(k_flux<T, 40, 3, false>);
            else
                prf ? go(k_flux<T, 20, 3, true>) : go(k_flux<T, 20, 3, false>);
        } else {
            if (stage == 1)
                prf ? go(k_flux<T, 40, 2, true>) : go(k_flux<T, 40, 2, false>);
            else
                prf ? go(k_flux<T, 20, 2, true>) : go(k_flux<T, 20, 2, false>);
        }
    } else {
        if (stage == 1)
            k_flux_single<T, 40><<<grid, 3 * FLUX_FACES, 0, s>>>(m, ph, W, poly, rec, ctrl, dt_override);
        else
            k_flux_single<T, 20><<<grid, 3 * FLUX_FACES, 0, s>>>(m, ph, W, poly, rec, ctrl, dt_override);
    }
    return cudaGetLastError();
}


template cudaError_t Launch<double>::flux(const DevMesh<double>&, const HostPhys&, const double*, const double*,
                                          double*, const double*, double, int, cudaStream_t, int);
template cudaError_t Launch<float>::flux(const DevMesh<float>&, const HostPhys&, const float*, const float*,
                                         float*, const double*, double, int, cudaStream_t, int);

}  // namespace gks
