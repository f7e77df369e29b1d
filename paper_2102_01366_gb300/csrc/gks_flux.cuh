// gks_flux.cuh -- the FP32 face flux of one block of faces (Sec. 2.2, 3,
// 4.4, 4.5), shared by the standalone flux kernel and the persistent stage
// kernel.
#pragma once

#include <cuda_runtime.h>

#include "gks_cells.cuh"
#include "gks_device.cuh"
#include "gks_face.cuh"
#include "gks_kernels.h"

namespace gks {

// Face flux with 6 threads per face: 3 Gauss points x 2 sides.  The two sides
// of a Gauss point sit in different warps (warps 0-2 left, 3-5 right) so that
// no warp diverges on the side; the interface equilibrium, its slopes and the
// partial outputs are exchanged through shared memory:
//   phase 1  own side: state at the point, face frame, slopes, rho <psi>+-
//   phase 2  W^c, collision times; own kinetic part; rho <a_i psi>+-
//   phase 3  right warps form the equilibrium slopes (once per point) and
//            share a^c, while in stage 1 the left warps form W^c relative to
//            the mean of the two cell averages (for the gradient records);
//            then left warps add the C2 (a^c.u) flux terms, right warps the
//            C1, C3 flux terms and the dW term
//   phase 4  left warps finish the flux entries, right warps the gradient
//            entries of the record; the 3 points of each face are summed.
constexpr int FP_GP = 3 * FLUX_FACES;  // Gauss points per block (96)

// FP32 stage-1 records carry 10 more entries: the face's reference flux
// (dt / 2) A F_n(W_m), formed in FP64, as FP32 hi and lo parts
template <int NR>
constexpr int rec_stride() { return NR == 40 ? REC1_F32 : NR; }

template <typename T, int NR>
struct FluxSmem {
    T w0[2][FP_GP][5];   // rho <psi>+- of each side
    T p[2][FP_GP];       // pressure of each side
    T dwc[2][FP_GP][15]; // rho <a_i psi>+- of each side
    T ac[NR == 40 ? 1 : FP_GP][15];  // stage 2: equilibrium slopes a^c_i (formed once, by the right warps)
    T out[2][FP_GP][20]; // partial Fh, D, W0, dW of each side
    T red[FP_GP * rec_stride<NR>()];  // weighted record entries per Gauss point
    // stage 1: each side's cell average (hi, lo) and R - average at the point
    // (phase 1); from phase 3 the left side's R - average slots hold W^c - W_m
    // (global frame)
    T dv[NR == 40 ? 2 : 1][NR == 40 ? FP_GP : 1][15];
    // stage 1: each side's half-space rho-moment <u^0> (erfc of its s), whose
    // erf the interface deviation reuses
    T m0[NR == 40 ? 2 : 1][NR == 40 ? FP_GP : 1];
};

// The two warps that hold the two sides of the same 32 Gauss points (warp w
// and warp w + 3) exchange through shared memory only with each other, so
// they meet at a named barrier of their own instead of the whole block's.
__device__ __forceinline__ void pair_barrier(int g, int base = 1) {
    asm volatile("bar.sync %0, %1;" ::"r"(base + (g >> 5)), "r"(64) : "memory");
}


// Stage 1, FP32: the interface state W^c of Eq. new-equ-part relative to W_m,
// the mean of the two cells' averages (the interior cell's average on a
// boundary face), in the global frame, into the left side's dv slot.  The
// gradient records sum w W(0) n over a cell's faces, where the O(|W|) parts
// cancel to |Omega| grad W; an FP32 W^c would leave its rounding, eps |W|,
// in each face term, i.e. an error ~ eps |W| / dr in the gradient.  Taken
// relative to W_m (exact differences of the hi / lo averages) and by the
// half-difference rules, W^c - W_m carries rounding relative to itself only.
// Interior and open faces; wall and fixed faces subtract directly.
template <typename T>
__device__ __forceinline__ void interface_deviation(T (*dv)[FP_GP][15], const T (*m0)[FP_GP], int g, int L, int Rc,
                                                    const T (*Rm)[3], const T (*w0)[FP_GP][5], T gm1) {
    T out[5];
    const bool pair = (L >= 0 || L == FLR_OPEN) && (Rc >= 0 || Rc == FLR_OPEN);
    if (pair) {
        T Wl[5], Wr[5], hg[5], sg[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const T D = T(0.5) * ((dv[0][g][q] - dv[1][g][q]) + (dv[0][g][5 + q] - dv[1][g][5 + q]));
            const T dl = D + dv[0][g][10 + q], dr = dv[1][g][10 + q] - D;
            hg[q] = T(0.5) * (dl - dr);
            sg[q] = T(0.5) * (dl + dr);
            Wl[q] = dv[0][g][q] + dv[0][g][10 + q];
            Wr[q] = dv[1][g][q] + dv[1][g][10 + q];
        }
        T tl[5] = {Wl[0], 0, 0, 0, Wl[4]}, tr[5] = {Wr[0], 0, 0, 0, Wr[4]}, th[5] = {hg[0], 0, 0, 0, hg[4]};
        rotate_vec(Rm, Wl + 1, tl + 1);
        rotate_vec(Rm, Wr + 1, tr + 1);
        rotate_vec(Rm, hg + 1, th + 1);
        // erf of each side's s from its half-space moment <u^0> (phase 1):
        // 2 <u^0>_{u1>0} - 1 on the left, 1 - 2 <u^0>_{u1<0} on the right
        psi_half_difference(tl, tr, th, gm1, T(2) * m0[0][g] - T(1), T(1) - T(2) * m0[1][g], out);
        to_global(Rm, out);
#pragma unroll
        for (int q = 0; q < 5; ++q) out[q] += sg[q];
    } else {
        const int in = L >= 0 ? 0 : 1;
#pragma unroll
        for (int q = 0; q < 5; ++q) out[q] = w0[0][g][q] + w0[1][g][q];
        to_global(Rm, out);
#pragma unroll
        for (int q = 0; q < 5; ++q) out[q] = (out[q] - dv[in][g][q]) - dv[in][g][5 + q];
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) dv[0][g][10 + q] = out[q];
}

// Stage 1, FP32: F_n(W^c) - F_n(W_m) (global frame) for the flux entries of
// the record, which hold the interface flux relative to the flux of W_m:
// over a cell's faces the O(|F|) parts cancel to |Omega| div F, and an FP32
// flux would leave eps |F| in each face term (an error ~ eps |W| per step in
// the averages, seen by the next stage's reconstruction as ~ eps |W| / h in
// the slopes).  W^c - W_m (phase 3) enters through the half-difference rules
// on interior and open faces; wall and fixed faces subtract directly.
template <typename T>
__device__ __forceinline__ void face_flux_deviation(const T (*dv)[FP_GP][15], int g, int L, int Rc,
                                                    const T (*Rm)[3], const T* Wcl, const T* n, T gm1, T* dF) {
    T Wc[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) Wc[q] = Wcl[q];
    to_global(Rm, Wc);
    const bool pair = (L >= 0 || L == FLR_OPEN) && (Rc >= 0 || Rc == FLR_OPEN);
    if (pair) {
        T Wm[5], h[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            Wm[q] = T(0.5) * (dv[0][g][q] + dv[1][g][q]);
            h[q] = T(0.5) * dv[0][g][10 + q];
        }
        normal_flux_half_difference(Wc, Wm, h, n, gm1, dF);
#pragma unroll
        for (int q = 0; q < 5; ++q) dF[q] *= T(2);
    } else {
        const int in = L >= 0 ? 0 : 1;
        T Wm[5], Fc[5], Fm[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) Wm[q] = dv[in][g][q] + dv[in][g][5 + q];
        normal_flux(Wc, n, gm1, Fc);
        normal_flux(Wm, n, gm1, Fm);
#pragma unroll
        for (int q = 0; q < 5; ++q) dF[q] = Fc[q] - Fm[q];
    }
}

// One block of FLUX_FACES faces (block index fb) by 2 FP_GP threads (tid):
// sm its shared memory, pair_base the first of the three named barriers of
// its side pairs, grp_id / 2 FP_GP the barrier of all its threads (0: the
// whole thread block).  The standalone kernel and the persistent stage
// kernel both run it.  XW: the mesh may have isothermal or moving wall
// faces (their ghosts are compiled only into those instances).
template <typename T, int NR, bool PRF, bool XW = true>
__device__ __forceinline__ void flux_faces(const DevMesh<T>& m, const Phys<T>& ph, const T* __restrict__ Wavg,
                                           const T* __restrict__ poly, T* __restrict__ rec,
                                           const double* __restrict__ ctrl, double dt_override, int64_t fb,
                                           int tid, FluxSmem<T, NR>& sm, int pair_base, int grp_id) {
    const int side = tid >= FP_GP ? 1 : 0;
    const int g = tid - side * FP_GP;  // Gauss point within the block
    const int lf = g / 3;
    const int k = g - 3 * lf;
    const int64_t f0 = fb * FLUX_FACES + lf;
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
    constexpr int XSR = Stride<T>::xs;
    const int mine = side == 0 ? L : Rc;
    const bool wall = mine == FLR_SLIP_WALL || mine == FLR_NOSLIP_WALL ||
                      (XW && (mine == FLR_ISOTHERMAL_WALL || mine == FLR_MOVING_WALL));
    T Ws[5], gs[3][5];
    // stage 1: the average this side refers to and R - average at the point
    T ahi[5], alo[5], dev[5];
    if (mine >= 0 || wall) {
        // a wall side starts from the interior cell's value at the point
        const int src = mine >= 0 ? side : 1 - side;
        const int64_t cell = mine >= 0 ? mine : (side == 0 ? Rc : L);
        const T X[3] = {geo[4 + 9 * src + 3 * k], geo[5 + 9 * src + 3 * k], geo[6 + 9 * src + 3 * k]};
        eval_poly(poly + cell * Stride<T>::poly, X, Ws, gs, dev, ahi, alo);
    } else {
        const int64_t in = side == 0 ? Rc : L;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            ahi[q] = Wavg[in * XSR + q];
            alo[q] = Wavg[in * XSR + XLO + q];
            dev[q] = T(0);
        }
        if (mine == FLR_FIXED) {
            const int src = 1 - side;
            const T X[3] = {geo[4 + 9 * src + 3 * k], geo[5 + 9 * src + 3 * k], geo[6 + 9 * src + 3 * k]};
            fixed_ghost(m.fixed + in * XSR, X, Ws, gs);
        } else {
            // open boundary: the missing side is the interior cell's average
            // with zero gradient (zeroth-order extrapolation; the paper leaves
            // outflow boundaries open, and copying the interior Gauss-point
            // state is not stable)
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                Ws[q] = ahi[q];
                gs[0][q] = gs[1][q] = gs[2][q] = T(0);
            }
        }
    }
    if constexpr (NR == 40) {
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            sm.dv[side][g][q] = ahi[q];
            sm.dv[side][g][5 + q] = alo[q];
            sm.dv[side][g][10 + q] = dev[q];
        }
    }
    T Rm[3][3];
    face_frame(n, Rm);
    T tW[5], tg[3][5];
    to_local(Rm, Ws, gs, tW, tg);
    if (mine == FLR_SLIP_WALL) slip_wall_ghost(tW, tg);
    if (mine == FLR_NOSLIP_WALL) noslip_wall_ghost(tW, tg);
    if constexpr (XW) {
        if (mine == FLR_ISOTHERMAL_WALL) isothermal_wall_ghost(tW, tg, ph.gm1, ph.twall);
        if (mine == FLR_MOVING_WALL) {
            T Uw[3];
            rotate_vec(Rm, ph.uwall, Uw);
            moving_wall_ghost(tW, tg, ph.gm1, Uw);
        }
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
    if constexpr (NR == 40) sm.m0[side][g] = t.u[0];
    pair_barrier(g, pair_base);

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
        // stage 1: the zeroth moments sum to W^c, which the record takes
        // relative to the mean of the two averages (phase 3); W0 keeps the
        // tau terms only
        if (NR != 40) axpy5(T(1), mw0, W0);
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
    pair_barrier(g, pair_base);

    // ---- phase 3 ----
    // Stage 1: the left warps form W^c - W_m (the gradient records' interface
    // state) while the right warps take all of the equilibrium part, the
    // a^c.u flux terms included, so the pair need not meet here; stage 2:
    // the left warps take the a^c.u terms after the right warps share a^c.
    constexpr bool RIGHT_GRAD = (NR == 40);
    {
        if (side == 1 || !RIGHT_GRAD) make_tab(t, C, ph.K, 0);
        T ac[3][5], divF[5];
        T mf1r[5] = {T(0), T(0), T(0), T(0), T(0)};
        if (side == 1) {
            // the equilibrium slopes, once per point (Eq. co for g^c)
            T dWc[3][5];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int q = 0; q < 5; ++q) dWc[i][q] = sm.dwc[0][g][5 * i + q] + sm.dwc[1][g][5 * i + q];
            const T ir = T(1) / C.rho;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                T b[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) b[q] = dWc[i][q] * ir;
                micro_slope(C, ph.K, b, ac[i]);
            }
            // rho sum_i <(a_i . psi) u_i psi> = sum_i d F_i / d x_i: the
            // equilibrium's moments differentiated along x_i are its Euler
            // fluxes' derivatives (Eq. co), taken here through the flux
            // Jacobians, which FP32 evaluates without the cancellation of the
            // fourth- and fifth-order velocity moments
            euler_divergence(C, Wc, ph.gm1, dWc, divF);
            if (RIGHT_GRAD) {
                acc_grad<1>(t, ac, C.rho, mf1r);
            } else {
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int q = 0; q < 5; ++q) sm.ac[g][5 * i + q] = ac[i][q];
            }
        } else if constexpr (NR == 40) {
            // the left warps meanwhile: stage 1's W^c - W_m for the gradient records
            interface_deviation(sm.dv, sm.m0, g, L, Rc, Rm, sm.w0, ph.gm1);
        }
        if (!RIGHT_GRAD || PRF) pair_barrier(g, pair_base);
        // Pr fix: the state integrals move to this side's (now unused) slope
        // slots; the right side adds the equilibrium part below
        T IW[10];
        if (PRF) {
#pragma unroll
            for (int q = 0; q < 10; ++q) IW[q] = sm.out[side][g][q];
        }
        if (side == 0) {
            if (!RIGHT_GRAD) {
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
            }
        } else {
            if (RIGHT_GRAD) {
                if (ph.smooth) {
                    axpy5(-tau * T(0.5) * dt, mf1r, Fh);
                } else {
                    axpy5(tc.q2, mf1r, Fh);
                    axpy5(tc.dq2, mf1r, D);
                }
            }
            T mf0[5] = {0}, mf2[5], mw1[5], dtW[5];
            acc_psi<1, 0, 0>(t, C.rho, mf0);
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                mw1[q] = divF[q];   // rho sum_i <(a_i . psi) u_i psi> (Eq. co)
                dtW[q] = -divF[q];  // rho <A psi>: the compatibility condition
            }
            // rho <u1 (A . psi) psi> = d F_1 / d t = J_1(W^c) rho <A psi>
            euler_flux_jvp(C, Wc, ph.gm1, 0, dtW, mf2);
            if (ph.smooth) {
                const T hd = T(0.5) * dt;
                // stage 1: hd F(W^c) joins the record in phase 4, relative to W_m
                if (NR != 40) axpy5(hd, mf0, Fh);
                axpy5(T(0.5) * hd * hd - tau * hd, mf2, Fh);
                axpy5(T(0.25) * dt * dt, mf2, D);
#pragma unroll
                for (int q = 0; q < 5; ++q) W0[q] = NR == 40 ? T(0) : Wc[q];  // tau terms cancel: <(a.u + A) psi> = 0
                axpy5(-dt, mw1, dWt);
                if (PRF) {
#pragma unroll
                    for (int q = 0; q < 5; ++q) {
                        IW[q] += hd * Wc[q] - T(0.5) * hd * hd * mw1[q];
                        IW[5 + q] += -T(0.25) * dt * dt * mw1[q];
                    }
                }
            } else {
                // q1 = dt / 2 - k0; stage 1 keeps -k0 here and takes (dt / 2) F(W^c)
                // relative to W_m in phase 4
                axpy5(NR == 40 ? -tc.k0 : tc.q1, mf0, Fh);
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
    pair_barrier(g, pair_base);

    // ---- phase 4: left warps the flux entries, right warps the gradient entries
    constexpr int RS = rec_stride<NR>();
    T* mine_rec = sm.red + g * RS;
    if (side == 0) {
        T Fs[5], Ds[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            Fs[q] = sm.out[0][g][q] + sm.out[1][g][q];
            Ds[q] = sm.out[0][g][5 + q] + sm.out[1][g][5 + q];
        }
        T Wcl[5];  // W^c, face frame
#pragma unroll
        for (int q = 0; q < 5; ++q) Wcl[q] = sm.w0[0][g][q] + sm.w0[1][g][q];
        if (PRF) {
            T IWh[5], IWd[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                IWh[q] = sm.dwc[0][g][q] + sm.dwc[1][g][q];
                IWd[q] = sm.dwc[0][g][5 + q] + sm.dwc[1][g][5 + q];
            }
            const T U[3] = {Wcl[1] / Wcl[0], Wcl[2] / Wcl[0], Wcl[3] / Wcl[0]};
            if constexpr (NR == 40) {
                // the Pr fix acts on the whole flux: put back (dt / 2) F_1(W^c)
                // for it and keep only its change of the energy entry
                const Prim<T> Cc = to_prim(Wcl, ph.gm1);
                const T F1c[5] = {Wcl[1], Wcl[1] * Cc.u + Cc.p, Wcl[1] * Cc.v, Wcl[1] * Cc.w, (Wcl[4] + Cc.p) * Cc.u};
                T Ff[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) Ff[q] = Fs[q] + T(0.5) * dt * F1c[q];
                const T before = Ff[4];
                prandtl_fix(ph.prf, U, IWh, Ff);
                Fs[4] += Ff[4] - before;
            } else {
                prandtl_fix(ph.prf, U, IWh, Fs);
            }
            prandtl_fix(ph.prf, U, IWd, Ds);
        }
        to_global(Rm, Fs);
        to_global(Rm, Ds);
        if constexpr (NR == 40) {
            // (dt / 2) (F_n(W^c) - F_n(W_m)): the flux of the interface state
            // relative to that of the mean of the two cell averages, whose
            // own flux, (dt / 2) A F_n(W_m), the record carries in FP64 terms
            T dF[5];
            face_flux_deviation(sm.dv, g, L, Rc, Rm, Wcl, n, ph.gm1, dF);
#pragma unroll
            for (int q = 0; q < 5; ++q) Fs[q] += T(0.5) * dt * dF[q];
            // once per face (its first Gauss point): the reference flux with
            // W_m from the hi / lo averages and the face's area vector A n
            // taken exactly (its sum over a closed cell vanishes to FP64
            // rounding, where the FP32 weights and normals leave eps A), in
            // FP32 pairs, stored as hi and lo parts; entering both cells with
            // opposite signs, it keeps the update exactly conservative
            F2 ref[5] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            if (k == 0) {
                F2 Wm[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    const F2 a = f2_add({sm.dv[0][g][q], sm.dv[0][g][5 + q]}, {sm.dv[1][g][q], sm.dv[1][g][5 + q]});
                    Wm[q] = {0.5f * a.hi, 0.5f * a.lo};
                }
                const float* an = m.fan + 6 * f;
                const F2 A[3] = {{an[0], an[1]}, {an[2], an[3]}, {an[4], an[5]}};
                const F2 mn = f2_add(f2_add(f2_mul(Wm[1], A[0]), f2_mul(Wm[2], A[1])), f2_mul(Wm[3], A[2]));
                const F2 un = f2_div(mn, Wm[0]);  // A u.n
                const F2 mm = f2_add(f2_add(f2_mul(Wm[1], Wm[1]), f2_mul(Wm[2], Wm[2])), f2_mul(Wm[3], Wm[3]));
                const F2 ke = f2_div(f2_scale(0.5f, mm), Wm[0]);
                const F2 pm = f2_scale((float)ph.gm1, f2_add(Wm[4], {-ke.hi, -ke.lo}));
                const float hd = 0.5f * (float)dt;
                ref[0] = f2_scale(hd, mn);
#pragma unroll
                for (int j = 0; j < 3; ++j) ref[1 + j] = f2_scale(hd, f2_add(f2_mul(Wm[1 + j], un), f2_mul(pm, A[j])));
                ref[4] = f2_scale(hd, f2_mul(f2_add(Wm[4], pm), un));
            }
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                mine_rec[REC1_REF + q] = ref[q].hi;
                mine_rec[REC1_REF + 5 + q] = ref[q].lo;
            }
        }
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
        if constexpr (NR == 40) {
            // W(0) - W_m: the tau terms plus W^c - W_m from phase 3
#pragma unroll
            for (int q = 0; q < 5; ++q) Zs[q] += sm.dv[0][g][10 + q];
        }
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
    group_barrier(grp_id, 2 * FP_GP);
    // sum the three Gauss points of each face; coalesced record store
    const int64_t base = fb * FLUX_FACES;
    for (int idx = tid; idx < FLUX_FACES * RS; idx += 2 * FP_GP) {
        const int fl = idx / RS, j = idx - fl * RS;
        if (base + fl < m.nf) {
            const T* r = sm.red + fl * 3 * RS + j;
            rec[(base + fl) * RS + j] = (r[0] + r[RS]) + r[2 * RS];
        }
    }
}


template <typename T>
inline Phys<T> make_phys(const HostPhys& p) {
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

// the FP32 face-flux launch on a mesh with isothermal or moving wall faces
// (the instances with their ghosts, in a translation unit of their own)
cudaError_t launch_flux_xw(const DevMesh<float>& m, const Phys<float>& ph, const float* W, const float* poly,
                           float* rec, const double* ctrl, double dt_override, int stage, cudaStream_t s,
                           int variant, bool prf);

// the face-flux kernel (6 threads per face): FLUX_FACES faces per block;
// MINB resident blocks per SM; PRF the Pr fix; XW isothermal / moving walls
template <typename T, int NR, int MINB, bool PRF, bool XW>
__global__ void __launch_bounds__(2 * FP_GP, MINB) k_flux(DevMesh<T> m, Phys<T> ph,
                                                     const T* __restrict__ Wavg,
                                                     const T* __restrict__ poly,
                                                     T* __restrict__ rec,
                                                     const double* __restrict__ ctrl,
                                                     double dt_override) {
    __shared__ FluxSmem<T, NR> sm;
    flux_faces<T, NR, PRF, XW>(m, ph, Wavg, poly, rec, ctrl, dt_override, blockIdx.x, threadIdx.x, sm, 1, 0);
}


}  // namespace gks
