// gks_point_adj.cuh -- reverse-mode (adjoint) derivative of the kinetic
// solution at one Gauss point, FP64, inviscid or viscous.
//
// gks_point_adj recomputes the forward quantities of gks_point (the two
// half-space moment tables, the interface equilibrium, the time coefficients,
// the micro-slopes of both sides and of the equilibrium, and with viscosity
// each side's time slope A from its full table) and then carries the
// output adjoints (of Fh, D, W0, dW) back through each of them in reverse
// order: every building block of gks_device.cuh has its transpose here
// (adj_*).  The moment sums are multilinear in the tables' one-dimensional
// moments; their adjoints go through adj_G, which distributes the adjoint of
// one product <u^P><v^Q><w^R> over its three factors.
#pragma once

#include "gks_device.cuh"

namespace gks {

using TabD = Tab<double>;

__device__ __forceinline__ void tab_zero(TabD& t) {
    for (int k = 0; k < 7; ++k) t.u[k] = t.v[k] = t.w[k] = 0.0;
    t.xi2 = t.xi4 = 0.0;
}

// adjoint of G = u[P] v[Q] w[R]
template <int P, int Q, int R>
__device__ __forceinline__ void adj_G(const TabD& t, TabD& lt, double lam) {
    lt.u[P] += lam * t.v[Q] * t.w[R];
    lt.v[Q] += lam * t.u[P] * t.w[R];
    lt.w[R] += lam * t.u[P] * t.v[Q];
}

// adjoint of Em<P,Q,R> = (G(P+2) + G(Q+2) + G(R+2) + xi2 G) / 2
template <int P, int Q, int R>
__device__ __forceinline__ void adj_E(const TabD& t, TabD& lt, double lam) {
    const double h = 0.5 * lam;
    adj_G<P + 2, Q, R>(t, lt, h);
    adj_G<P, Q + 2, R>(t, lt, h);
    adj_G<P, Q, R + 2>(t, lt, h);
    adj_G<P, Q, R>(t, lt, h * t.xi2);
    lt.xi2 += h * Gm<P, Q, R>(t);
}

// adjoint of E2m<P,Q,R>
template <int P, int Q, int R>
__device__ __forceinline__ void adj_E2(const TabD& t, TabD& lt, double lam) {
    const double q = 0.25 * lam;
    adj_G<P + 4, Q, R>(t, lt, q);
    adj_G<P, Q + 4, R>(t, lt, q);
    adj_G<P, Q, R + 4>(t, lt, q);
    adj_G<P, Q, R>(t, lt, q * t.xi4);
    lt.xi4 += q * Gm<P, Q, R>(t);
    adj_G<P + 2, Q + 2, R>(t, lt, 2.0 * q);
    adj_G<P + 2, Q, R + 2>(t, lt, 2.0 * q);
    adj_G<P, Q + 2, R + 2>(t, lt, 2.0 * q);
    adj_G<P + 2, Q, R>(t, lt, 2.0 * q * t.xi2);
    adj_G<P, Q + 2, R>(t, lt, 2.0 * q * t.xi2);
    adj_G<P, Q, R + 2>(t, lt, 2.0 * q * t.xi2);
    lt.xi2 += 2.0 * q * (Gm<P + 2, Q, R>(t) + Gm<P, Q + 2, R>(t) + Gm<P, Q, R + 2>(t));
}

// adjoint of acc_psi<P,Q,R>(t, c, out): out += c <psi u^P v^Q w^R>
template <int P, int Q, int R>
__device__ __forceinline__ void adj_acc_psi(const TabD& t, double c, const double* lo, TabD& lt, double& lc) {
    lc += lo[0] * Gm<P, Q, R>(t) + lo[1] * Gm<P + 1, Q, R>(t) + lo[2] * Gm<P, Q + 1, R>(t) +
          lo[3] * Gm<P, Q, R + 1>(t) + lo[4] * Em<P, Q, R>(t);
    adj_G<P, Q, R>(t, lt, c * lo[0]);
    adj_G<P + 1, Q, R>(t, lt, c * lo[1]);
    adj_G<P, Q + 1, R>(t, lt, c * lo[2]);
    adj_G<P, Q, R + 1>(t, lt, c * lo[3]);
    adj_E<P, Q, R>(t, lt, c * lo[4]);
}

// adjoint of acc_apsi<P,Q,R>(t, a, c, out): out_k += sum_j c a_j M_kj with the
// symmetric moment matrix M_kj = <psi_k psi_j u^P v^Q w^R>
template <int P, int Q, int R>
__device__ __forceinline__ void adj_acc_apsi(const TabD& t, const double* a, double c, const double* lo,
                                             TabD& lt, double* la, double& lc) {
    double M[5][5];
    M[0][0] = Gm<P, Q, R>(t);
    M[0][1] = M[1][0] = Gm<P + 1, Q, R>(t);
    M[0][2] = M[2][0] = Gm<P, Q + 1, R>(t);
    M[0][3] = M[3][0] = Gm<P, Q, R + 1>(t);
    M[0][4] = M[4][0] = Em<P, Q, R>(t);
    M[1][1] = Gm<P + 2, Q, R>(t);
    M[1][2] = M[2][1] = Gm<P + 1, Q + 1, R>(t);
    M[1][3] = M[3][1] = Gm<P + 1, Q, R + 1>(t);
    M[1][4] = M[4][1] = Em<P + 1, Q, R>(t);
    M[2][2] = Gm<P, Q + 2, R>(t);
    M[2][3] = M[3][2] = Gm<P, Q + 1, R + 1>(t);
    M[2][4] = M[4][2] = Em<P, Q + 1, R>(t);
    M[3][3] = Gm<P, Q, R + 2>(t);
    M[3][4] = M[4][3] = Em<P, Q, R + 1>(t);
    M[4][4] = E2m<P, Q, R>(t);
    double ca[5];
    for (int j = 0; j < 5; ++j) ca[j] = c * a[j];
    for (int j = 0; j < 5; ++j) {
        double s = 0.0;
        for (int k = 0; k < 5; ++k) s += lo[k] * M[k][j];
        la[j] += c * s;
        lc += a[j] * s;
    }
    // adjoint of each distinct entry: lo_k ca_j + lo_j ca_k off the diagonal
    auto e = [&](int k, int j) { return k == j ? lo[k] * ca[k] : lo[k] * ca[j] + lo[j] * ca[k]; };
    adj_G<P, Q, R>(t, lt, e(0, 0));
    adj_G<P + 1, Q, R>(t, lt, e(0, 1));
    adj_G<P, Q + 1, R>(t, lt, e(0, 2));
    adj_G<P, Q, R + 1>(t, lt, e(0, 3));
    adj_E<P, Q, R>(t, lt, e(0, 4));
    adj_G<P + 2, Q, R>(t, lt, e(1, 1));
    adj_G<P + 1, Q + 1, R>(t, lt, e(1, 2));
    adj_G<P + 1, Q, R + 1>(t, lt, e(1, 3));
    adj_E<P + 1, Q, R>(t, lt, e(1, 4));
    adj_G<P, Q + 2, R>(t, lt, e(2, 2));
    adj_G<P, Q + 1, R + 1>(t, lt, e(2, 3));
    adj_E<P, Q + 1, R>(t, lt, e(2, 4));
    adj_G<P, Q, R + 2>(t, lt, e(3, 3));
    adj_E<P, Q, R + 1>(t, lt, e(3, 4));
    adj_E2<P, Q, R>(t, lt, e(4, 4));
}

// adjoint of acc_grad<P>(t, a, c, out)
template <int P>
__device__ __forceinline__ void adj_acc_grad(const TabD& t, const double (*a)[5], double c, const double* lo,
                                             TabD& lt, double (*la)[5], double& lc) {
    adj_acc_apsi<P + 1, 0, 0>(t, a[0], c, lo, lt, la[0], lc);
    adj_acc_apsi<P, 1, 0>(t, a[1], c, lo, lt, la[1], lc);
    adj_acc_apsi<P, 0, 1>(t, a[2], c, lo, lt, la[2], lc);
}

// adjoints of a primitive state, in the fields of Prim
struct PrimAdj {
    double rho = 0.0, u = 0.0, v = 0.0, w = 0.0, lam = 0.0, p = 0.0;
};

// adjoint of the moment recursion m[k+2] = U m[k+1] + (k+1) h m[k]
__device__ __forceinline__ void adj_recur(const double* m, double U, double h, double* lm, double& lU,
                                          double& lh) {
    for (int k = 4; k >= 0; --k) {
        const double l = lm[k + 2];
        lU += l * m[k + 1];
        lm[k + 1] += l * U;
        lh += l * (double)(k + 1) * m[k];
        lm[k] += l * (double)(k + 1) * h;
    }
}

// adjoint of make_tab(t, s, K, half): the table's adjoint lt into the state's
__device__ __forceinline__ void adj_make_tab(const TabD& t, const Prim<double>& s, double K, int half,
                                             const TabD& lt, PrimAdj& ls) {
    const double h = 0.5 / s.lam;
    double lh = K * lt.xi2 + 2.0 * (K * K + 2.0 * K) * h * lt.xi4;
    double lu[7], lv[7], lw[7];
    for (int k = 0; k < 7; ++k) {
        lu[k] = lt.u[k];
        lv[k] = lt.v[k];
        lw[k] = lt.w[k];
    }
    adj_recur(t.u, s.u, h, lu, ls.u, lh);
    adj_recur(t.v, s.v, h, lv, ls.v, lh);
    adj_recur(t.w, s.w, h, lw, ls.w, lh);
    ls.v += lv[1];
    ls.w += lw[1];
    if (half == 0) {
        ls.u += lu[1];
    } else {
        const double sg = half > 0 ? 1.0 : -1.0;
        const double sl = sqrt(s.lam);
        const double e = exp(-s.lam * s.u * s.u);
        const double c = 0.5 * 0.56418958354775628695;  // 1 / (2 sqrt(pi))
        // u1 = U u0 + sg c e / sl
        ls.u += lu[1] * t.u[0];
        lu[0] += lu[1] * s.u;
        ls.u += lu[1] * sg * c * e * (-2.0 * s.lam * s.u) / sl;
        ls.lam += lu[1] * sg * c * e * (-s.u * s.u / sl - 0.5 / (s.lam * sl));
        // u0 = erfc(x) / 2 with x = -sg sl U;  d erfc / dx = -2/sqrt(pi) exp(-x^2)
        const double du0dx = -0.56418958354775628695 * e;
        ls.u += lu[0] * du0dx * (-sg * sl);
        ls.lam += lu[0] * du0dx * (-sg * s.u * 0.5 / sl);
    }
    ls.lam += lh * (-0.5 / (s.lam * s.lam));
}

// adjoint of to_prim(W, gm1): the primitive adjoint ls into lW
__device__ __forceinline__ void adj_to_prim(const double* W, double gm1, const Prim<double>& s,
                                            const PrimAdj& ls, double* lW) {
    double lp = ls.p, lrho = ls.rho;
    lrho += ls.lam * 0.5 / s.p;
    lp += ls.lam * (-0.5 * s.rho / (s.p * s.p));
    double lu = ls.u, lv = ls.v, lw = ls.w;
    lW[4] += gm1 * lp;
    lW[1] += -0.5 * gm1 * lp * s.u;
    lW[2] += -0.5 * gm1 * lp * s.v;
    lW[3] += -0.5 * gm1 * lp * s.w;
    lu += -0.5 * gm1 * lp * W[1];
    lv += -0.5 * gm1 * lp * W[2];
    lw += -0.5 * gm1 * lp * W[3];
    const double ir = 1.0 / W[0];
    lW[1] += lu * ir;
    lW[2] += lv * ir;
    lW[3] += lw * ir;
    const double lir = lu * W[1] + lv * W[2] + lw * W[3];
    lW[0] += lrho - lir * ir * ir;
}

// adjoint of micro_slope(s, K, b, a): la into ls and lb
__device__ __forceinline__ void adj_micro_slope(const Prim<double>& s, double K, const double* b,
                                                const double* la_in, PrimAdj& ls, double* lb) {
    // forward
    const double q = s.u * s.u + s.v * s.v + s.w * s.w;
    const double e = q + (K + 3.0) * 0.5 / s.lam;
    const double r1 = b[1] - s.u * b[0], r2 = b[2] - s.v * b[0], r3 = b[3] - s.w * b[0];
    const double r4 = 2.0 * b[4] - e * b[0];
    const double kap = 4.0 * s.lam * s.lam / (K + 3.0);
    const double S = s.u * r1 + s.v * r2 + s.w * r3;
    const double a4 = kap * (r4 - 2.0 * S);
    const double tl = 2.0 * s.lam;
    const double a1 = tl * r1 - s.u * a4, a2 = tl * r2 - s.v * a4, a3 = tl * r3 - s.w * a4;
    // reverse
    double la1 = la_in[1], la2 = la_in[2], la3 = la_in[3], la4 = la_in[4];
    const double la0 = la_in[0];
    double le = 0.0, ltl = 0.0, lr1 = 0.0, lr2 = 0.0, lr3 = 0.0, lr4 = 0.0;
    // a0 = b0 - u a1 - v a2 - w a3 - a4 e / 2
    lb[0] += la0;
    ls.u += -la0 * a1;
    la1 += -la0 * s.u;
    ls.v += -la0 * a2;
    la2 += -la0 * s.v;
    ls.w += -la0 * a3;
    la3 += -la0 * s.w;
    la4 += -0.5 * la0 * e;
    le += -0.5 * la0 * a4;
    // a_i = tl r_i - u_i a4
    ltl += la1 * r1 + la2 * r2 + la3 * r3;
    lr1 += la1 * tl;
    lr2 += la2 * tl;
    lr3 += la3 * tl;
    ls.u += -la1 * a4;
    ls.v += -la2 * a4;
    ls.w += -la3 * a4;
    la4 += -(la1 * s.u + la2 * s.v + la3 * s.w);
    ls.lam += 2.0 * ltl;
    // a4 = kap (r4 - 2 S)
    const double lkap = la4 * (r4 - 2.0 * S);
    lr4 += la4 * kap;
    const double lS = -2.0 * kap * la4;
    ls.u += lS * r1;
    ls.v += lS * r2;
    ls.w += lS * r3;
    lr1 += lS * s.u;
    lr2 += lS * s.v;
    lr3 += lS * s.w;
    ls.lam += lkap * 8.0 * s.lam / (K + 3.0);
    // r4 = 2 b4 - e b0, r_i = b_i - u_i b0
    lb[4] += 2.0 * lr4;
    le += -lr4 * b[0];
    lb[0] += -lr4 * e - lr1 * s.u - lr2 * s.v - lr3 * s.w;
    lb[1] += lr1;
    lb[2] += lr2;
    lb[3] += lr3;
    ls.u += -lr1 * b[0];
    ls.v += -lr2 * b[0];
    ls.w += -lr3 * b[0];
    // e = q + (K + 3) / (2 lam)
    ls.lam += le * (-(K + 3.0) * 0.5 / (s.lam * s.lam));
    ls.u += 2.0 * s.u * le;
    ls.v += 2.0 * s.v * le;
    ls.w += 2.0 * s.w * le;
}

// Adjoint of gks_point: output adjoints lFh, lD, lW0, ldW (face frame) into
// the input adjoints lWl, lgl, lWr, lgr (accumulated).  Inviscid (tau = 0)
// and viscous (tau = mu / p_c, with the A terms of each side) alike; VISC
// must equal ph.viscous (the inviscid instance keeps no viscous state).
template <bool VISC>
__device__ void gks_point_adj(const Phys<double>& ph, const double* Wl, const double (*gl)[5],
                              const double* Wr, const double (*gr)[5], double dt, const double* lFh_out,
                              const double* lD_out, const double* lW0, const double* ldW, double* lWl,
                              double (*lgl)[5], double* lWr, double (*lgr)[5]) {
    const double K = ph.K;
    constexpr bool visc = VISC;
    const bool smooth = ph.smooth != 0;
    const double* Win[2] = {Wl, Wr};
    const double (*gin[2])[5] = {gl, gr};
    // ---- forward recomputation ----
    Prim<double> P[2];
    TabD th[2];
    double Wc[5] = {0, 0, 0, 0, 0};
    for (int s = 0; s < 2; ++s) {
        P[s] = to_prim(Win[s], ph.gm1);
        make_tab(th[s], P[s], K, s == 0 ? +1 : -1);
        acc_psi<0, 0, 0>(th[s], P[s].rho, Wc);
    }
    const Prim<double> C = to_prim(Wc, ph.gm1);
    const TimeCoef<double> tc = time_coefs(ph, P[0].p, P[1].p, C.p, dt);
    const double tau = tc.tau;
    double a[2][3][5], As[2][5], rs[2][5];
    double dWc[3][5] = {};
    TabD tfs[2];  // full tables of the two sides (viscous only)
    for (int s = 0; s < 2; ++s) {
        const double ir = 1.0 / P[s].rho;
        for (int i = 0; i < 3; ++i) {
            double b[5];
            for (int k = 0; k < 5; ++k) b[k] = gin[s][i][k] * ir;
            micro_slope(P[s], K, b, a[s][i]);
            acc_apsi<0, 0, 0>(th[s], a[s][i], P[s].rho, dWc[i]);
        }
        if (visc && !smooth) {
            make_tab(tfs[s], P[s], K, 0);
            for (int k = 0; k < 5; ++k) rs[s][k] = 0.0;
            acc_grad<0>(tfs[s], a[s], -1.0, rs[s]);
            micro_slope(P[s], K, rs[s], As[s]);
        }
    }
    TabD tf;
    make_tab(tf, C, K, 0);
    double ac[3][5], Ac[5], rA[5], bc[3][5];
    for (int i = 0; i < 3; ++i) {
        for (int k = 0; k < 5; ++k) bc[i][k] = dWc[i][k] / C.rho;
        micro_slope(C, K, bc[i], ac[i]);
    }
    for (int k = 0; k < 5; ++k) rA[k] = 0.0;
    acc_grad<0>(tf, ac, -1.0, rA);
    micro_slope(C, K, rA, Ac);
    const double hd = 0.5 * dt;
    // equilibrium sums (recomputed for the coefficient adjoints)
    double mf0[5] = {0, 0, 0, 0, 0}, mf1[5] = {0, 0, 0, 0, 0}, mf2[5] = {0, 0, 0, 0, 0}, mw1[5];
    acc_psi<1, 0, 0>(tf, C.rho, mf0);
    acc_grad<1>(tf, ac, C.rho, mf1);
    acc_apsi<1, 0, 0>(tf, Ac, C.rho, mf2);
    for (int k = 0; k < 5; ++k) mw1[k] = -C.rho * rA[k];

    // ---- reverse ----
    // Pr fix (viscous): F_E += prf (qf - U1 qw) on Fh and D, with
    // qf = F_E - U.F_m + |U|^2/2 F_rho, qw the same of the state integral IW
    // and U = U^c.  Its transpose turns the output adjoints into those of the
    // uncorrected Fh, D, of IWh, IWd and of U^c.
    double lFh[5], lD[5], lIWh[5] = {0, 0, 0, 0, 0}, lIWd[5] = {0, 0, 0, 0, 0}, lU[3] = {0, 0, 0};
    for (int k = 0; k < 5; ++k) {
        lFh[k] = lFh_out[k];
        lD[k] = lD_out[k];
    }
    const bool prfix = VISC && ph.prf != 0.0;
    if (prfix) {
        // forward: the uncorrected Fh, D and the state integrals IWh, IWd
        double F[2][5], IW[2][5];
        for (int k = 0; k < 5; ++k) {
            if (smooth) {
                F[0][k] = hd * mf0[k] - tau * hd * mf1[k] + (0.5 * hd * hd - tau * hd) * mf2[k];
                F[1][k] = 0.25 * dt * dt * mf2[k];
                IW[0][k] = hd * Wc[k] - 0.5 * hd * hd * mw1[k];
                IW[1][k] = -0.25 * dt * dt * mw1[k];
            } else {
                F[0][k] = tc.q1 * mf0[k] + tc.q2 * mf1[k] + tc.q3 * mf2[k];
                F[1][k] = tc.dq1 * mf0[k] + tc.dq2 * mf1[k] + tc.dq3 * mf2[k];
                IW[0][k] = tc.q1 * Wc[k] + (tc.q2 - tc.q3) * mw1[k];
                IW[1][k] = tc.dq1 * Wc[k] + (tc.dq2 - tc.dq3) * mw1[k];
            }
        }
        if (!smooth)
            for (int s = 0; s < 2; ++s) {
                double kf0[5] = {0, 0, 0, 0, 0}, kf1[5] = {0, 0, 0, 0, 0}, kf2[5] = {0, 0, 0, 0, 0},
                       kw0[5] = {0, 0, 0, 0, 0}, kw1[5] = {0, 0, 0, 0, 0}, kw2[5] = {0, 0, 0, 0, 0};
                acc_psi<1, 0, 0>(th[s], P[s].rho, kf0);
                acc_grad<1>(th[s], a[s], P[s].rho, kf1);
                acc_apsi<1, 0, 0>(th[s], As[s], P[s].rho, kf2);
                acc_psi<0, 0, 0>(th[s], P[s].rho, kw0);
                acc_grad<0>(th[s], a[s], P[s].rho, kw1);
                acc_apsi<0, 0, 0>(th[s], As[s], P[s].rho, kw2);
                for (int k = 0; k < 5; ++k) {
                    F[0][k] += tc.k0 * kf0[k] - (tau * tc.k0 + tc.k1) * kf1[k] - tau * tc.k0 * kf2[k];
                    F[1][k] += tc.dk0 * kf0[k] - (tau * tc.dk0 + tc.dk1) * kf1[k] - tau * tc.dk0 * kf2[k];
                    IW[0][k] += tc.k0 * kw0[k] - (tau * tc.k0 + tc.k1) * kw1[k] - tau * tc.k0 * kw2[k];
                    IW[1][k] += tc.dk0 * kw0[k] - (tau * tc.dk0 + tc.dk1) * kw1[k] - tau * tc.dk0 * kw2[k];
                }
            }
        const double U[3] = {C.u, C.v, C.w};
        const double uu = 0.5 * (U[0] * U[0] + U[1] * U[1] + U[2] * U[2]);
        const double gq[5] = {uu, -U[0], -U[1], -U[2], 1.0};  // d q / d (F or IW)
        for (int h = 0; h < 2; ++h) {
            double* lF = h == 0 ? lFh : lD;
            double* lIW = h == 0 ? lIWh : lIWd;
            const double l = ph.prf * lF[4];
            const double qw = IW[h][4] - (U[0] * IW[h][1] + U[1] * IW[h][2] + U[2] * IW[h][3]) + uu * IW[h][0];
            for (int j = 0; j < 3; ++j)
                lU[j] += l * (-F[h][1 + j] + U[j] * F[h][0] - (j == 0 ? qw : 0.0) -
                              U[0] * (-IW[h][1 + j] + U[j] * IW[h][0]));
            for (int k = 0; k < 5; ++k) {
                lF[k] += l * gq[k];
                lIW[k] += -U[0] * l * gq[k];
            }
        }
    }
    TabD ltf;
    tab_zero(ltf);
    PrimAdj lC;
    lC.u += lU[0];
    lC.v += lU[1];
    lC.w += lU[2];
    double lCrho = 0.0;  // adjoint of the rho factor of the equilibrium sums
    double lWc[5] = {0, 0, 0, 0, 0};
    double lac[3][5] = {}, lAc[5] = {0, 0, 0, 0, 0}, lrA[5] = {0, 0, 0, 0, 0};
    // adjoints of the time coefficients and of tau
    double lk0 = 0, lk1 = 0, ldk0 = 0, ldk1 = 0, lq1 = 0, lq2 = 0, lq3 = 0, ldq1 = 0, ldq2 = 0, ldq3 = 0;
    double lE = 0, ltau = 0;
    double lmf0[5], lmf1[5], lmf2[5], lmw1[5];
    if (smooth) {
        for (int k = 0; k < 5; ++k) {
            lmf0[k] = hd * lFh[k];
            lmf1[k] = -tau * hd * lFh[k];
            lmf2[k] = (0.5 * hd * hd - tau * hd) * lFh[k] + 0.25 * dt * dt * lD[k];
            lmw1[k] = -dt * ldW[k];
            lWc[k] += lW0[k];
            ltau += -hd * lFh[k] * (mf1[k] + mf2[k]);
            // Pr fix: IWh = hd W^c - hd^2/2 mw1, IWd = -dt^2/4 mw1
            lWc[k] += hd * lIWh[k];
            lmw1[k] += -0.5 * hd * hd * lIWh[k] - 0.25 * dt * dt * lIWd[k];
        }
    } else {
        const double C23 = dt * (tc.E - 1.0);
        for (int k = 0; k < 5; ++k) {
            lmf0[k] = tc.q1 * lFh[k] + tc.dq1 * lD[k];
            lmf1[k] = tc.q2 * lFh[k] + tc.dq2 * lD[k];
            lmf2[k] = tc.q3 * lFh[k] + tc.dq3 * lD[k];
            lmw1[k] = C23 * ldW[k];
            lq1 += lFh[k] * mf0[k];
            lq2 += lFh[k] * mf1[k];
            lq3 += lFh[k] * mf2[k];
            ldq1 += lD[k] * mf0[k];
            ldq2 += lD[k] * mf1[k];
            ldq3 += lD[k] * mf2[k];
            lE += dt * ldW[k] * mw1[k];
            // Pr fix: IWh = q1 W^c + (q2 - q3) mw1, IWd with the d-coefficients
            lWc[k] += tc.q1 * lIWh[k] + tc.dq1 * lIWd[k];
            lmw1[k] += (tc.q2 - tc.q3) * lIWh[k] + (tc.dq2 - tc.dq3) * lIWd[k];
            lq1 += lIWh[k] * Wc[k];
            lq2 += lIWh[k] * mw1[k];
            lq3 -= lIWh[k] * mw1[k];
            ldq1 += lIWd[k] * Wc[k];
            ldq2 += lIWd[k] * mw1[k];
            ldq3 -= lIWd[k] * mw1[k];
        }
    }
    // mw1 = -rho_c rA
    for (int k = 0; k < 5; ++k) {
        lCrho += -lmw1[k] * rA[k];
        lrA[k] += -C.rho * lmw1[k];
    }
    adj_acc_apsi<1, 0, 0>(tf, Ac, C.rho, lmf2, ltf, lAc, lCrho);
    adj_acc_grad<1>(tf, ac, C.rho, lmf1, ltf, lac, lCrho);
    adj_acc_psi<1, 0, 0>(tf, C.rho, lmf0, ltf, lCrho);
    adj_micro_slope(C, K, rA, lAc, lC, lrA);
    {
        double lunused = 0.0;
        adj_acc_grad<0>(tf, ac, -1.0, lrA, ltf, lac, lunused);
    }
    double ldWc[3][5] = {};
    for (int i = 0; i < 3; ++i) {
        double lb[5] = {0, 0, 0, 0, 0};
        adj_micro_slope(C, K, bc[i], lac[i], lC, lb);
        for (int k = 0; k < 5; ++k) {
            ldWc[i][k] += lb[k] / C.rho;
            lC.rho += -lb[k] * dWc[i][k] / (C.rho * C.rho);
        }
    }
    adj_make_tab(tf, C, K, 0, ltf, lC);
    lC.rho += lCrho;

    // the two sides: kinetic parts (full flux), their sums, slopes and tables
    TabD lth[2];
    PrimAdj lP[2];
    double la[2][3][5] = {};
    for (int s = 0; s < 2; ++s) {
        tab_zero(lth[s]);
        double lrho = 0.0, lA[5] = {0, 0, 0, 0, 0};
        if (!smooth) {
            double kf0[5] = {0, 0, 0, 0, 0}, kf1[5] = {0, 0, 0, 0, 0}, kw0[5] = {0, 0, 0, 0, 0},
                   kw1[5] = {0, 0, 0, 0, 0}, kf2[5] = {0, 0, 0, 0, 0}, kw2[5] = {0, 0, 0, 0, 0};
            acc_psi<1, 0, 0>(th[s], P[s].rho, kf0);
            acc_grad<1>(th[s], a[s], P[s].rho, kf1);
            acc_psi<0, 0, 0>(th[s], P[s].rho, kw0);
            acc_grad<0>(th[s], a[s], P[s].rho, kw1);
            if (visc) {
                acc_apsi<1, 0, 0>(th[s], As[s], P[s].rho, kf2);
                acc_apsi<0, 0, 0>(th[s], As[s], P[s].rho, kw2);
            }
            double lkf0[5], lkf1[5], lkw0[5], lkw1[5], lkf2[5], lkw2[5];
            const double cw1 = tau - (tau + dt) * tc.E, cw2 = tau * (1.0 - tc.E);
            for (int k = 0; k < 5; ++k) {
                // Fh += k0 f0 - (tau k0 + k1) f1 - tau k0 f2; D alike with dk;
                // W0 += w0 - tau w1 - tau w2; dW += cw1 w1 + cw2 w2
                lkf0[k] = tc.k0 * lFh[k] + tc.dk0 * lD[k];
                lkf1[k] = -(tau * tc.k0 + tc.k1) * lFh[k] - (tau * tc.dk0 + tc.dk1) * lD[k];
                lkf2[k] = -tau * tc.k0 * lFh[k] - tau * tc.dk0 * lD[k];
                lkw0[k] = lW0[k];
                lkw1[k] = -tau * lW0[k] + cw1 * ldW[k];
                lkw2[k] = -tau * lW0[k] + cw2 * ldW[k];
                lk0 += lFh[k] * (kf0[k] - tau * kf1[k] - tau * kf2[k]);
                lk1 += -lFh[k] * kf1[k];
                ldk0 += lD[k] * (kf0[k] - tau * kf1[k] - tau * kf2[k]);
                ldk1 += -lD[k] * kf1[k];
                ltau += -lFh[k] * tc.k0 * (kf1[k] + kf2[k]) - lD[k] * tc.dk0 * (kf1[k] + kf2[k]) -
                        lW0[k] * (kw1[k] + kw2[k]) + ldW[k] * ((1.0 - tc.E) * (kw1[k] + kw2[k]));
                lE += ldW[k] * (-(tau + dt) * kw1[k] - tau * kw2[k]);
                // Pr fix: this side's part of IWh, IWd (k- and dk-coefficients)
                lkw0[k] += tc.k0 * lIWh[k] + tc.dk0 * lIWd[k];
                lkw1[k] += -(tau * tc.k0 + tc.k1) * lIWh[k] - (tau * tc.dk0 + tc.dk1) * lIWd[k];
                lkw2[k] += -tau * tc.k0 * lIWh[k] - tau * tc.dk0 * lIWd[k];
                lk0 += lIWh[k] * (kw0[k] - tau * kw1[k] - tau * kw2[k]);
                lk1 -= lIWh[k] * kw1[k];
                ldk0 += lIWd[k] * (kw0[k] - tau * kw1[k] - tau * kw2[k]);
                ldk1 -= lIWd[k] * kw1[k];
                ltau += -(lIWh[k] * tc.k0 + lIWd[k] * tc.dk0) * (kw1[k] + kw2[k]);
            }
            adj_acc_psi<1, 0, 0>(th[s], P[s].rho, lkf0, lth[s], lrho);
            adj_acc_grad<1>(th[s], a[s], P[s].rho, lkf1, lth[s], la[s], lrho);
            adj_acc_psi<0, 0, 0>(th[s], P[s].rho, lkw0, lth[s], lrho);
            adj_acc_grad<0>(th[s], a[s], P[s].rho, lkw1, lth[s], la[s], lrho);
            if (visc) {
                adj_acc_apsi<1, 0, 0>(th[s], As[s], P[s].rho, lkf2, lth[s], lA, lrho);
                adj_acc_apsi<0, 0, 0>(th[s], As[s], P[s].rho, lkw2, lth[s], lA, lrho);
            }
        }
        if (visc && !smooth) {
            // A = micro_slope(P, K, r), r = -sum_i <(a_i . psi) u_i psi> over the full table
            double lr[5] = {0, 0, 0, 0, 0}, lunused = 0.0;
            TabD ltfs;
            tab_zero(ltfs);
            adj_micro_slope(P[s], K, rs[s], lA, lP[s], lr);
            adj_acc_grad<0>(tfs[s], a[s], -1.0, lr, ltfs, la[s], lunused);
            adj_make_tab(tfs[s], P[s], K, 0, ltfs, lP[s]);
        }
        for (int i = 0; i < 3; ++i) adj_acc_apsi<0, 0, 0>(th[s], a[s][i], P[s].rho, ldWc[i], lth[s], la[s][i], lrho);
        double (*lg)[5] = s == 0 ? lgl : lgr;
        const double ir = 1.0 / P[s].rho;
        for (int i = 0; i < 3; ++i) {
            double b[5], lb[5] = {0, 0, 0, 0, 0};
            for (int k = 0; k < 5; ++k) b[k] = gin[s][i][k] * ir;
            adj_micro_slope(P[s], K, b, la[s][i], lP[s], lb);
            for (int k = 0; k < 5; ++k) {
                lg[i][k] += lb[k] * ir;
                lrho += -lb[k] * gin[s][i][k] * ir * ir;
            }
        }
        lP[s].rho += lrho;
    }
    // time coefficients -> tau_n, tau -> the pressures
    if (!smooth) {
        // q1 = hd - k0; q2 = k1 + tau k0 - tau hd; q3 = hd^2/2 - tau hd + tau k0;
        // dq1 = tn omh^2; dq2 = dk1 + tau dk0; dq3 = dt^2/4 + tau dk0
        lk0 += -lq1 + tau * lq2 + tau * lq3;
        lk1 += lq2;
        ltau += (tc.k0 - hd) * (lq2 + lq3) + tc.dk0 * (ldq2 + ldq3);
        ldk1 += ldq2;
        ldk0 += tau * (ldq2 + ldq3);
        const double tn = tc.tau_n;
        const double Eh = sqrt(tc.E);
        const double omh = 1.0 - Eh;
        double ltn = 0.0, lEh = 0.0, lomh = 0.0;
        ltn += lk0 * omh;
        lomh += lk0 * tn;
        ltn += lk1 * (2.0 * tn * omh - hd * Eh);
        lomh += lk1 * tn * tn;
        lEh += lk1 * (-tn * hd);
        ltn += ldk0 * (-omh * omh);
        lomh += ldk0 * (-2.0 * tn * omh);
        ltn += ldk1 * (-2.0 * tn * omh * omh + dt * Eh * omh);
        lomh += ldk1 * (-2.0 * tn * tn * omh + tn * dt * Eh);
        lEh += ldk1 * tn * dt * omh;
        ltn += ldq1 * omh * omh;
        lomh += ldq1 * 2.0 * tn * omh;
        lEh += 2.0 * Eh * lE - lomh;
        ltn += lEh * Eh * hd / (tn * tn);
        // tn = (viscous ? tau : tau_eps dt) + tau_c |x| dt, x = (pl - pr) / (pl + pr)
        if (visc) ltau += ltn;
        const double pl = P[0].p, pr = P[1].p;
        const double x = (pl - pr) / (pl + pr);
        const double sx = x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0);
        const double lx = ltn * ph.tau_c * dt * sx;
        const double den = (pl + pr) * (pl + pr);
        lP[0].p += lx * 2.0 * pr / den;
        lP[1].p += lx * (-2.0 * pl) / den;
    }
    // tau = mu / p_c (viscous)
    if (visc) lC.p += -ltau * ph.mu / (C.p * C.p);
    adj_to_prim(Wc, ph.gm1, C, lC, lWc);
    for (int s = 0; s < 2; ++s) adj_acc_psi<0, 0, 0>(th[s], P[s].rho, lWc, lth[s], lP[s].rho);
    for (int s = 0; s < 2; ++s) {
        adj_make_tab(th[s], P[s], K, s == 0 ? +1 : -1, lth[s], lP[s]);
        adj_to_prim(Win[s], ph.gm1, P[s], lP[s], s == 0 ? lWl : lWr);
    }
}

}  // namespace gks
