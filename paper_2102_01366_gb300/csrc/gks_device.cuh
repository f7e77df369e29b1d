// gks_device.cuh -- device-side building blocks of libgks, templated on the
// working precision T (double: FP64 path; float: FP32-bulk path).
//
//   * Maxwellian moments <u^p v^q w^r> over the full space or a half space
//     (Sec. 2.2; the half-space zeroth and first moments come from erfc and
//     the Gaussian tail, higher ones from the standard recursion);
//   * micro-slopes a = a_1 + a_2 u + a_3 v + a_4 w + a_5 (u^2+xi^2)/2 solving
//     <a psi> = dW / rho (Eq. co) in closed form (the inverse of the 5x5
//     moment matrix of a Maxwellian);
//   * the time-dependent kinetic solution at one Gauss point in the face
//     frame (Eq. 2nd-flux / Eq. 2nd-smooth-flux with the equilibrium state
//     of Eq. new-equ-part): time integrals of the flux over [0, dt/2] and
//     [0, dt], and the interface states at t = 0 and t = dt.
#pragma once

#include <cstdint>

namespace gks {

// --------------------------------------------------------------- math --
__device__ __forceinline__ double d_exp(double x) { return exp(x); }
__device__ __forceinline__ float d_exp(float x) { return expf(x); }
__device__ __forceinline__ double d_erfc(double x) { return erfc(x); }
__device__ __forceinline__ float d_erfc(float x) { return erfcf(x); }
__device__ __forceinline__ double d_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float d_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double d_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float d_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double d_abs(double x) { return fabs(x); }
__device__ __forceinline__ float d_abs(float x) { return fabsf(x); }
__device__ __forceinline__ double d_cbrt(double x) { return cbrt(x); }
__device__ __forceinline__ float d_cbrt(float x) { return cbrtf(x); }

// |x|^(4/3) as x * cbrt(x) for x >= 0
template <typename T>
__device__ __forceinline__ T pow43(T x) { return x * d_cbrt(x); }

// Error-free transformation of a sum (Knuth's TwoSum): a + b = s + e exactly.
template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T& s, T& e) {
    s = a + b;
    T bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Compensated accumulator: value = hi + lo.
template <typename T>
struct CSum {
    T hi, lo;
    __device__ __forceinline__ void init() { hi = T(0); lo = T(0); }
    __device__ __forceinline__ void add(T x) {
        T s, e;
        two_sum(hi, x, s, e);
        hi = s;
        lo += e;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// ------------------------------------------------------------ params --
template <typename T>
struct Phys {
    T gamma, gm1, K;     // K internal degrees of freedom
    T tau_eps, tau_c, mu;
    T eps_w;
    T prf;               // Pr fix: 1/Pr - 1 (0 without it)
    T twall;             // temperature p / rho of isothermal walls
    T uwall[3];          // velocity of moving walls (global frame)
    int viscous, smooth;
};

// ------------------------------------------------------- Maxwellian --
template <typename T>
struct Prim {
    T rho, u, v, w, lam, p;
};

template <typename T>
__device__ __forceinline__ Prim<T> to_prim(const T* W, T gm1) {
    Prim<T> s;
    s.rho = W[0];
    T ir = T(1) / W[0];
    s.u = W[1] * ir;
    s.v = W[2] * ir;
    s.w = W[3] * ir;
    s.p = gm1 * (W[4] - T(0.5) * (W[1] * s.u + W[2] * s.v + W[3] * s.w));
    s.lam = T(0.5) * s.rho / s.p;
    return s;
}

// normalised moments <u^k> (k < 7) for u (full or half space), v, w and
// <xi^2>, <xi^4>
template <typename T>
struct Tab {
    T u[7], v[7], w[7];
    T xi2, xi4;
};

template <typename T>
__device__ __forceinline__ void mom_recur(T* m, T U, T h) {
    // h = 1 / (2 lambda); <u^(k+2)> = U <u^(k+1)> + (k+1) h <u^k>
#pragma unroll
    for (int k = 0; k < 5; ++k) m[k + 2] = U * m[k + 1] + T(k + 1) * h * m[k];
}

// half: +1 restricts u > 0, -1 restricts u < 0, 0 is the whole space
template <typename T>
__device__ __forceinline__ void make_tab(Tab<T>& t, const Prim<T>& s, T K, int half) {
    const T h = T(0.5) / s.lam;
    if (half == 0) {
        t.u[0] = T(1);
        t.u[1] = s.u;
    } else {
        const T sg = half > 0 ? T(1) : T(-1);
        const T sl = d_sqrt(s.lam);
        t.u[0] = T(0.5) * d_erfc(-sg * sl * s.u);
        // Gaussian tail term exp(-lam U^2) / (2 sqrt(pi lam))
        const T inv_sqrt_pi = T(0.56418958354775628695);
        t.u[1] = s.u * t.u[0] + sg * T(0.5) * inv_sqrt_pi * d_exp(-s.lam * s.u * s.u) / sl;
    }
    mom_recur(t.u, s.u, h);
    t.v[0] = T(1);
    t.v[1] = s.v;
    mom_recur(t.v, s.v, h);
    t.w[0] = T(1);
    t.w[1] = s.w;
    mom_recur(t.w, s.w, h);
    t.xi2 = K * h;
    t.xi4 = (K * K + T(2) * K) * h * h;
}

// only the u-moments change between the full space and a half space
template <typename T>
__device__ __forceinline__ void make_half_u(Tab<T>& t, const Prim<T>& s, int half) {
    const T h = T(0.5) / s.lam;
    const T sg = half > 0 ? T(1) : T(-1);
    const T sl = d_sqrt(s.lam);
    t.u[0] = T(0.5) * d_erfc(-sg * sl * s.u);
    const T inv_sqrt_pi = T(0.56418958354775628695);
    t.u[1] = s.u * t.u[0] + sg * T(0.5) * inv_sqrt_pi * d_exp(-s.lam * s.u * s.u) / sl;
    mom_recur(t.u, s.u, h);
}

template <int P, int Q, int R, typename T>
__device__ __forceinline__ T Gm(const Tab<T>& t) {
    return t.u[P] * t.v[Q] * t.w[R];
}

// <eps u^P v^Q w^R>, eps = (u^2 + v^2 + w^2 + xi^2) / 2
template <int P, int Q, int R, typename T>
__device__ __forceinline__ T Em(const Tab<T>& t) {
    return T(0.5) * (Gm<P + 2, Q, R>(t) + Gm<P, Q + 2, R>(t) + Gm<P, Q, R + 2>(t) + t.xi2 * Gm<P, Q, R>(t));
}

// <eps^2 u^P v^Q w^R>
template <int P, int Q, int R, typename T>
__device__ __forceinline__ T E2m(const Tab<T>& t) {
    return T(0.25) * (Gm<P + 4, Q, R>(t) + Gm<P, Q + 4, R>(t) + Gm<P, Q, R + 4>(t) + t.xi4 * Gm<P, Q, R>(t) +
                      T(2) * (Gm<P + 2, Q + 2, R>(t) + Gm<P + 2, Q, R + 2>(t) + Gm<P, Q + 2, R + 2>(t)) +
                      T(2) * t.xi2 * (Gm<P + 2, Q, R>(t) + Gm<P, Q + 2, R>(t) + Gm<P, Q, R + 2>(t)));
}

// out_alpha += c * <psi_alpha u^P v^Q w^R>
template <int P, int Q, int R, typename T>
__device__ __forceinline__ void acc_psi(const Tab<T>& t, T c, T* out) {
    out[0] += c * Gm<P, Q, R>(t);
    out[1] += c * Gm<P + 1, Q, R>(t);
    out[2] += c * Gm<P, Q + 1, R>(t);
    out[3] += c * Gm<P, Q, R + 1>(t);
    out[4] += c * Em<P, Q, R>(t);
}

// out_alpha += c * <psi_alpha (a.psi) u^P v^Q w^R>
template <int P, int Q, int R, typename T>
__device__ __forceinline__ void acc_apsi(const Tab<T>& t, const T* a, T c, T* out) {
    const T a0 = c * a[0], a1 = c * a[1], a2 = c * a[2], a3 = c * a[3], a4 = c * a[4];
    out[0] += a0 * Gm<P, Q, R>(t) + a1 * Gm<P + 1, Q, R>(t) + a2 * Gm<P, Q + 1, R>(t) +
              a3 * Gm<P, Q, R + 1>(t) + a4 * Em<P, Q, R>(t);
    out[1] += a0 * Gm<P + 1, Q, R>(t) + a1 * Gm<P + 2, Q, R>(t) + a2 * Gm<P + 1, Q + 1, R>(t) +
              a3 * Gm<P + 1, Q, R + 1>(t) + a4 * Em<P + 1, Q, R>(t);
    out[2] += a0 * Gm<P, Q + 1, R>(t) + a1 * Gm<P + 1, Q + 1, R>(t) + a2 * Gm<P, Q + 2, R>(t) +
              a3 * Gm<P, Q + 1, R + 1>(t) + a4 * Em<P, Q + 1, R>(t);
    out[3] += a0 * Gm<P, Q, R + 1>(t) + a1 * Gm<P + 1, Q, R + 1>(t) + a2 * Gm<P, Q + 1, R + 1>(t) +
              a3 * Gm<P, Q, R + 2>(t) + a4 * Em<P, Q, R + 1>(t);
    out[4] += a0 * Em<P, Q, R>(t) + a1 * Em<P + 1, Q, R>(t) + a2 * Em<P, Q + 1, R>(t) +
              a3 * Em<P, Q, R + 1>(t) + a4 * E2m<P, Q, R>(t);
}

// out += c * sum_i <psi (a_i . psi) u_i u^P>   (P = 0 or 1 extra powers of u)
template <int P, typename T>
__device__ __forceinline__ void acc_grad(const Tab<T>& t, const T (*a)[5], T c, T* out) {
    acc_apsi<P + 1, 0, 0>(t, a[0], c, out);
    acc_apsi<P, 1, 0>(t, a[1], c, out);
    acc_apsi<P, 0, 1>(t, a[2], c, out);
}

// Micro-slope of a Maxwellian: solves <a psi> = b (full space) for a, with
// the closed-form inverse of the moment matrix.
template <typename T>
__device__ __forceinline__ void micro_slope(const Prim<T>& s, T K, const T* b, T* a) {
    const T q = s.u * s.u + s.v * s.v + s.w * s.w;
    const T e = q + (K + T(3)) * T(0.5) / s.lam;  // 2 <eps>
    const T r1 = b[1] - s.u * b[0];
    const T r2 = b[2] - s.v * b[0];
    const T r3 = b[3] - s.w * b[0];
    const T r4 = T(2) * b[4] - e * b[0];
    const T a4 = T(4) * s.lam * s.lam / (K + T(3)) * (r4 - T(2) * (s.u * r1 + s.v * r2 + s.w * r3));
    const T tl = T(2) * s.lam;
    a[1] = tl * r1 - s.u * a4;
    a[2] = tl * r2 - s.v * a4;
    a[3] = tl * r3 - s.w * a4;
    a[4] = a4;
    a[0] = b[0] - s.u * a[1] - s.v * a[2] - s.w * a[3] - T(0.5) * a4 * e;
}

// Slopes a_x, a_y, a_z and A of a Maxwellian with conservative gradients
// g[i][q] (Eq. co): <a_i psi> = g_i / rho, <(A + sum_i a_i u_i) psi> = 0.
// r (may be NULL) receives <A psi> = -sum_i <(a_i . psi) u_i psi>, which
// the flux needs again (rho <A psi> is the W-rate of the equilibrium part).
template <typename T>
__device__ __forceinline__ void state_slopes(const Prim<T>& s, const Tab<T>& full, T K,
                                             const T (*g)[5], T (*a)[5], T* A, T* r_out = nullptr) {
    const T ir = T(1) / s.rho;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        T b[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) b[k] = g[i][k] * ir;
        micro_slope(s, K, b, a[i]);
    }
    T r[5] = {T(0), T(0), T(0), T(0), T(0)};
    acc_grad<0>(full, a, T(-1), r);
    micro_slope(s, K, r, A);
    if (r_out)
#pragma unroll
        for (int k = 0; k < 5; ++k) r_out[k] = r[k];
}

// Directional derivative of the Euler flux along x_dir (face frame) of the
// state W (primitives s): out = (d F_dir / d W) dW, with
// F_dir = (m_dir, m_j u_dir + p delta_j,dir, (E + p) u_dir) and
// p = (gamma - 1)(E - |m|^2 / (2 rho)).  For a Maxwellian g(W(x, t)), whose
// derivatives are g (a . psi) with rho <a psi> = dW (Eq. co), the velocity
// moments rho <u_dir (a . psi) psi> equal this product.
template <typename T>
__device__ __forceinline__ void euler_flux_jvp(const Prim<T>& s, const T* W, T gm1, int dir, const T* dW, T* out) {
    const T u[3] = {s.u, s.v, s.w};
    const T ud = u[dir];
    const T dp = gm1 * (dW[4] - (u[0] * dW[1] + u[1] * dW[2] + u[2] * dW[3]) +
                        T(0.5) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) * dW[0]);
    const T dud = (dW[1 + dir] - ud * dW[0]) / s.rho;
    out[0] = dW[1 + dir];
#pragma unroll
    for (int j = 0; j < 3; ++j) out[1 + j] = dW[1 + j] * ud + W[1 + j] * dud + (j == dir ? dp : T(0));
    out[4] = (dW[4] + dp) * ud + (W[4] + s.p) * dud;
}

// sum_i (d F_i / d W) g_i: the divergence of the Euler flux for the
// conservative gradients g[i][q] (face frame)
template <typename T>
__device__ __forceinline__ void euler_divergence(const Prim<T>& s, const T* W, T gm1, const T (*g)[5], T* out) {
#pragma unroll
    for (int q = 0; q < 5; ++q) out[q] = T(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        T d[5];
        euler_flux_jvp(s, W, gm1, i, g[i], d);
#pragma unroll
        for (int q = 0; q < 5; ++q) out[q] += d[q];
    }
}

// Time coefficients of Eq. 2nd-flux over [0, dt/2] (k0, k1 for the kinetic
// factors e and t e; q1..q3 for C1..C3) and their "dt minus twice dt/2"
// differences (dk*, dq*), with E = exp(-dt/tau_n) = Eh^2.
template <typename T>
struct TimeCoef {
    T tau, tau_n, E;
    T k0, k1, q1, q2, q3;
    T dk0, dk1, dq1, dq2, dq3;
};

template <typename T>
__device__ __forceinline__ TimeCoef<T> time_coefs(const Phys<T>& ph, T pl, T pr, T pc, T dt) {
    TimeCoef<T> c;
    c.tau = ph.viscous ? ph.mu / pc : T(0);
    const T jump = d_abs((pl - pr) / (pl + pr)) * dt;
    c.tau_n = (ph.viscous ? ph.mu / pc : ph.tau_eps * dt) + ph.tau_c * jump;
    const T hd = T(0.5) * dt;
    const T Eh = d_exp(-hd / c.tau_n);
    c.E = Eh * Eh;
    const T omh = T(1) - Eh;
    const T tn = c.tau_n, tau = c.tau;
    c.k0 = tn * omh;
    c.k1 = tn * (tn * omh - hd * Eh);
    c.q1 = hd - c.k0;
    c.q2 = c.k1 + tau * c.k0 - tau * hd;
    c.q3 = T(0.5) * hd * hd - tau * hd + tau * c.k0;
    c.dk0 = -tn * omh * omh;
    c.dk1 = -tn * tn * omh * omh + tn * dt * Eh * omh;
    c.dq1 = tn * omh * omh;
    c.dq2 = c.dk1 + tau * c.dk0;
    c.dq3 = T(0.25) * dt * dt + tau * c.dk0;
    return c;
}

template <typename T>
__device__ __forceinline__ void axpy5(T a, const T* x, T* y) {
#pragma unroll
    for (int k = 0; k < 5; ++k) y[k] += a * x[k];
}

// Pr fix of the energy flux over one time interval: F_E += (1/Pr - 1) q with
// q = int (u1 - U1) (|u - U|^2 + xi^2) / 2 f, expanded into the flux F and the
// state integral IW = int psi f over the same interval (U the interface
// equilibrium velocity, face frame):
//   q = F_E - U.F_m + |U|^2/2 F_rho - U1 (IW_E - U.IW_m + |U|^2/2 IW_rho)
template <typename T>
__device__ __forceinline__ void prandtl_fix(T prf, const T* U, const T* IW, T* F) {
    const T uu = T(0.5) * (U[0] * U[0] + U[1] * U[1] + U[2] * U[2]);
    const T qf = F[4] - (U[0] * F[1] + U[1] * F[2] + U[2] * F[3]) + uu * F[0];
    const T qw = IW[4] - (U[0] * IW[1] + U[1] * IW[2] + U[2] * IW[3]) + uu * IW[0];
    F[4] += prf * (qf - U[0] * qw);
}

// One side's initial-state (kinetic) part of Eq. 2nd-flux,
//   e^{-t/tau_n} g [1 - (tau + t) a.u - tau A] H(+-u1),
// added to Fh, D, W0, dW.  Each velocity moment is formed once and scaled by
// the time coefficients of all four outputs; the A terms carry a factor tau
// and are skipped for inviscid flow.  Also returns this side's contributions
// rho <psi> to W^c and rho <a_i psi> to its slopes (half space).
template <typename T>
__device__ __forceinline__ void kinetic_side(const Phys<T>& ph, const Prim<T>& S, const T (*g)[5], int half,
                                             Tab<T>& t, T (*a)[5], T* A) {
    const T ir = T(1) / S.rho;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        T b[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) b[k] = g[i][k] * ir;
        micro_slope(S, ph.K, b, a[i]);
    }
    if (ph.viscous) {
        make_tab(t, S, ph.K, 0);
        T r[5] = {T(0), T(0), T(0), T(0), T(0)};
        acc_grad<0>(t, a, T(-1), r);
        micro_slope(S, ph.K, r, A);
        make_half_u(t, S, half);
    } else {
        make_tab(t, S, ph.K, half);
    }
}

// Time-dependent kinetic solution at one Gauss point, face frame.
//   Wl, Wr: states; gl[i][q], gr[i][q]: gradients (direction i, comp q)
// Outputs, each 5 long:
//   Fh = int_0^{dt/2} F dt,  D = int_0^dt F dt - 2 Fh   (second-order part)
//   W0 = W(0),               dW = W(dt) - W(0)
// D and dW are formed from differences of the time coefficients, in which
// the leading terms cancel exactly, instead of by subtracting the rounded
// integrals (which loses about three digits in FP32).
template <typename T>
__device__ __forceinline__ void gks_point(const Phys<T>& ph, const T* Wl, const T (*gl)[5],
                                          const T* Wr, const T (*gr)[5], T dt, T* Fh, T* D,
                                          T* W0, T* dW) {
    const Prim<T> P[2] = {to_prim(Wl, ph.gm1), to_prim(Wr, ph.gm1)};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        Fh[k] = T(0);
        D[k] = T(0);
        W0[k] = T(0);
        dW[k] = T(0);
    }
    // W^c from the half-space moments of both sides (Eq. new-equ-part)
    T Wc[5] = {T(0), T(0), T(0), T(0), T(0)};
    {
        Tab<T> t;
        make_tab(t, P[0], ph.K, +1);
        acc_psi<0, 0, 0>(t, P[0].rho, Wc);
        make_tab(t, P[1], ph.K, -1);
        acc_psi<0, 0, 0>(t, P[1].rho, Wc);
    }
    const Prim<T> C = to_prim(Wc, ph.gm1);
    const TimeCoef<T> tc = time_coefs(ph, P[0].p, P[1].p, C.p, dt);
    const T tau = tc.tau;
    // state integrals over [0, dt/2] and their "dt minus twice" differences,
    // for the Pr fix only
    const bool prfix = ph.prf != T(0);
    T IWh[5], IWd[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) IWh[k] = IWd[k] = T(0);
    T dWc[3][5];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 5; ++k) dWc[i][k] = T(0);
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
        const Prim<T> S = P[side];
        Tab<T> t;
        T a[3][5], A[5];
        kinetic_side(ph, S, side == 0 ? gl : gr, side == 0 ? +1 : -1, t, a, A);
#pragma unroll
        for (int i = 0; i < 3; ++i) acc_apsi<0, 0, 0>(t, a[i], S.rho, dWc[i]);
        if (ph.smooth) continue;
        T mf0[5] = {0}, mf1[5] = {0}, mw0[5] = {0}, mw1[5] = {0};
        acc_psi<1, 0, 0>(t, S.rho, mf0);
        acc_grad<1>(t, a, S.rho, mf1);
        acc_psi<0, 0, 0>(t, S.rho, mw0);
        acc_grad<0>(t, a, S.rho, mw1);
        axpy5(tc.k0, mf0, Fh);
        axpy5(-(tau * tc.k0 + tc.k1), mf1, Fh);
        axpy5(tc.dk0, mf0, D);
        axpy5(-(tau * tc.dk0 + tc.dk1), mf1, D);
        axpy5(T(1), mw0, W0);
        axpy5(-tau, mw1, W0);
        axpy5(tau - (tau + dt) * tc.E, mw1, dW);
        if (prfix) {
            axpy5(tc.k0, mw0, IWh);
            axpy5(-(tau * tc.k0 + tc.k1), mw1, IWh);
            axpy5(tc.dk0, mw0, IWd);
            axpy5(-(tau * tc.dk0 + tc.dk1), mw1, IWd);
        }
        if (ph.viscous) {
            T mf2[5] = {0}, mw2[5] = {0};
            acc_apsi<1, 0, 0>(t, A, S.rho, mf2);
            acc_apsi<0, 0, 0>(t, A, S.rho, mw2);
            axpy5(-tau * tc.k0, mf2, Fh);
            axpy5(-tau * tc.dk0, mf2, D);
            axpy5(-tau, mw2, W0);
            axpy5(tau * (T(1) - tc.E), mw2, dW);
            if (prfix) {
                axpy5(-tau * tc.k0, mw2, IWh);
                axpy5(-tau * tc.dk0, mw2, IWd);
            }
        }
    }
    // hydrodynamic (equilibrium) part: C1 g^c + C2 a^c.u g^c + C3 A^c g^c
    Tab<T> t;
    make_tab(t, C, ph.K, 0);
    T ac[3][5], Ac[5], rA[5];
    state_slopes(C, t, ph.K, dWc, ac, Ac, rA);
    T mf0[5] = {0}, mf1[5] = {0}, mf2[5] = {0}, mw1[5];
    acc_psi<1, 0, 0>(t, C.rho, mf0);
    acc_grad<1>(t, ac, C.rho, mf1);
    acc_apsi<1, 0, 0>(t, Ac, C.rho, mf2);
#pragma unroll
    for (int k = 0; k < 5; ++k) mw1[k] = -C.rho * rA[k];  // rho sum_i <(a_i . psi) u_i psi> (Eq. co)
    if (ph.smooth) {
        // f = g^c - tau (a^c.u + A^c) g^c + A^c g^c t, Eq. 2nd-smooth-flux
        const T hd = T(0.5) * dt;
        axpy5(hd, mf0, Fh);
        axpy5(-tau * hd, mf1, Fh);
        axpy5(T(0.5) * hd * hd - tau * hd, mf2, Fh);
        axpy5(T(0.25) * dt * dt, mf2, D);
#pragma unroll
        for (int k = 0; k < 5; ++k) W0[k] = Wc[k];  // tau terms cancel: <(a.u + A) psi> = 0
        axpy5(-dt, mw1, dW);
        if (prfix) {
            // int psi f over [0, dt/2] = hd W^c - hd^2/2 rho <(a^c.u) psi> (the
            // A^c moments are minus the a^c.u ones); the difference -dt^2/4 of it
            axpy5(hd, Wc, IWh);
            axpy5(-T(0.5) * hd * hd, mw1, IWh);
            axpy5(-T(0.25) * dt * dt, mw1, IWd);
        }
    } else {
        axpy5(tc.q1, mf0, Fh);
        axpy5(tc.q2, mf1, Fh);
        axpy5(tc.q3, mf2, Fh);
        axpy5(tc.dq1, mf0, D);
        axpy5(tc.dq2, mf1, D);
        axpy5(tc.dq3, mf2, D);
        // t = dt: C2, C3 (C1 cancelled against the kinetic W0 terms)
        const T C2 = (dt + tau) * tc.E - tau, C3 = dt - tau + tau * tc.E;
        axpy5(C2 - C3, mw1, dW);
        if (prfix) {
            axpy5(tc.q1, Wc, IWh);
            axpy5(tc.q2 - tc.q3, mw1, IWh);
            axpy5(tc.dq1, Wc, IWd);
            axpy5(tc.dq2 - tc.dq3, mw1, IWd);
        }
    }
    if (prfix) {
        const T U[3] = {C.u, C.v, C.w};
        prandtl_fix(ph.prf, U, IWh, Fh);
        prandtl_fix(ph.prf, U, IWd, D);
    }
}


// --------------------------------------------- half differences --
// A quantity known on the two sides of a face: its values l, r and,
// accurate to the rounding of itself, its half-difference h = (l - r) / 2.
// The rules below are exact identities for finite differences (not
// linearisations), so h keeps its relative accuracy however small it is,
// where (l - r) / 2 formed from the rounded values would carry the rounding
// of l and r.  FP32 bulk uses them to form the interface state W^c
// (Eq. new-equ-part) relative to the mean of the two sides.
template <typename T>
struct HDiff {
    T l, r, h;
    __device__ __forceinline__ T mid() const { return T(0.5) * (l + r); }
};

template <typename T>
__device__ __forceinline__ HDiff<T> hd_add(const HDiff<T>& a, const HDiff<T>& b) {
    return {a.l + b.l, a.r + b.r, a.h + b.h};
}

template <typename T>
__device__ __forceinline__ HDiff<T> hd_scale(T c, const HDiff<T>& a) {
    return {c * a.l, c * a.r, c * a.h};
}

// (l_a l_b - r_a r_b) / 2 = h_a mid_b + mid_a h_b
template <typename T>
__device__ __forceinline__ HDiff<T> hd_mul(const HDiff<T>& a, const HDiff<T>& b) {
    return {a.l * b.l, a.r * b.r, a.h * b.mid() + a.mid() * b.h};
}

// (l_a / l_b - r_a / r_b) / 2 = (h_a mid_b - mid_a h_b) / (l_b r_b)
template <typename T>
__device__ __forceinline__ HDiff<T> hd_div(const HDiff<T>& a, const HDiff<T>& b) {
    return {a.l / b.l, a.r / b.r, (a.h * b.mid() - a.mid() * b.h) / (b.l * b.r)};
}

// (sqrt l - sqrt r) / 2 = h / (sqrt l + sqrt r)
template <typename T>
__device__ __forceinline__ HDiff<T> hd_sqrt(const HDiff<T>& a) {
    const T sl = d_sqrt(a.l), sr = d_sqrt(a.r);
    return {sl, sr, a.h / (sl + sr)};
}

// (e^{-l} - e^{-r}) / 2, factored on the larger exponential so that expm1
// stays within (-1, 0] (the other factoring overflows times underflows for
// far-apart arguments): -e^{-l} expm1(2 h) / 2 for h <= 0, e^{-r}
// expm1(-2 h) / 2 otherwise
__device__ __forceinline__ HDiff<float> hd_expneg(const HDiff<float>& a) {
    const float el = expf(-a.l), er = expf(-a.r);
    const float h = a.h <= 0.0f ? -0.5f * el * expm1f(2.0f * a.h) : 0.5f * er * expm1f(-2.0f * a.h);
    return {el, er, h};
}

// (erf l - erf r) / 2 = (1 / sqrt pi) int_r^l e^{-t^2} dt, given erf l and
// erf r (el, er).  For |l - r| <= 0.1 the integral is taken by 3-point and
// up to |l - r| <= 1 by 5-point Gauss-Legendre quadrature on [r, l] (errors
// below 1e-9 and 2e-8 of the integral at those lengths, far less for
// shorter intervals); for longer intervals the difference of the two
// complementary error functions of the tails, which does not cancel there.
__device__ __forceinline__ HDiff<float> hd_erf(const HDiff<float>& a, float el, float er) {
    float h;
    if (fabsf(a.h) <= 0.05f) {
        // nodes and weights of the 3-point Gauss-Legendre rule on [-1, 1]
        const float x1 = 0.77459666924148338f, w0 = 0.88888888888888889f, w1 = 0.55555555555555556f;
        const float m = a.mid(), d = a.h;
        auto g = [](float t) { return expf(-t * t); };
        h = 0.56418958354775628695f * d * (w0 * g(m) + w1 * (g(m + x1 * d) + g(m - x1 * d)));
    } else if (fabsf(a.h) <= 0.5f) {
        // nodes and weights of the 5-point Gauss-Legendre rule on [-1, 1]
        const float x1 = 0.53846931010568309f, x2 = 0.90617984593866399f;
        const float w0 = 0.56888888888888889f, w1 = 0.47862867049936647f, w2 = 0.23692688505618909f;
        const float m = a.mid(), d = a.h;
        auto g = [](float t) { return expf(-t * t); };
        const float sum = w0 * g(m) + w1 * (g(m + x1 * d) + g(m - x1 * d)) + w2 * (g(m + x2 * d) + g(m - x2 * d));
        h = 0.56418958354775628695f * d * sum;  // 1 / sqrt(pi)
    } else if (a.mid() > 0.0f) {
        h = 0.5f * (erfcf(a.r) - erfcf(a.l));
    } else {
        h = 0.5f * (erfcf(-a.l) - erfcf(-a.r));
    }
    return {el, er, h};
}

// Half-difference of psi(W) = rho <psi>_{u1>0} - rho <psi>_{u1<0} between
// the two states Wl, Wr (face frame, x1 along the normal), given the
// half-difference h of the states themselves and erf of each state's s
// (below).  With s = sqrt(lambda) U1 =
// W1 / sqrt(2 p rho), e0 = erf(s) and g = e^{-s^2} / sqrt(pi lambda) =
// e^{-s^2} sqrt(2 p / (pi rho)), the half-space moments of Sec. 2.2 give
//   psi(W) = (rho e0, W1 e0 + rho g, W2 e0, W3 e0, W4 e0 + W1 g / 2),
// and W^c = rho_l <psi>_{u1>0} + rho_r <psi>_{u1<0} = (Wl + Wr) / 2 +
// (psi(Wl) - psi(Wr)) / 2, so W^c minus the mean of the two states is h_psi.
__device__ __forceinline__ void psi_half_difference(const float* Wl, const float* Wr, const float* h, float gm1,
                                                    float erf_l, float erf_r, float* out) {
    const HDiff<float> rho{Wl[0], Wr[0], h[0]}, m1{Wl[1], Wr[1], h[1]}, m2{Wl[2], Wr[2], h[2]};
    const HDiff<float> m3{Wl[3], Wr[3], h[3]}, E{Wl[4], Wr[4], h[4]};
    const HDiff<float> mm = hd_add(hd_add(hd_mul(m1, m1), hd_mul(m2, m2)), hd_mul(m3, m3));
    const HDiff<float> p = hd_scale(gm1, hd_add(E, hd_scale(-0.5f, hd_div(mm, rho))));
    const HDiff<float> sy = hd_sqrt(hd_scale(2.0f, hd_mul(p, rho)));
    const HDiff<float> sv = hd_div(m1, sy);
    const HDiff<float> e0 = hd_erf(sv, erf_l, erf_r);
    const HDiff<float> ex = hd_expneg(hd_mul(sv, sv));
    const HDiff<float> g = hd_scale(0.79788456080286536f, hd_mul(ex, hd_sqrt(hd_div(p, rho))));  // sqrt(2 / pi)
    out[0] = hd_mul(rho, e0).h;
    out[1] = hd_mul(m1, e0).h + hd_mul(rho, g).h;
    out[2] = hd_mul(m2, e0).h;
    out[3] = hd_mul(m3, e0).h;
    out[4] = hd_mul(E, e0).h + 0.5f * hd_mul(m1, g).h;
}

// Normal Euler flux F_n(W) = (m.n, m u_n + p n, (E + p) u_n), u_n = m.n / rho,
// of a global-frame state.
__device__ __forceinline__ void normal_flux(const float* W, const float* n, float gm1, float* out) {
    const float mn = W[1] * n[0] + W[2] * n[1] + W[3] * n[2];
    const float un = mn / W[0];
    const float p = gm1 * (W[4] - 0.5f * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]) / W[0]);
    out[0] = mn;
#pragma unroll
    for (int j = 0; j < 3; ++j) out[1 + j] = W[1 + j] * un + p * n[j];
    out[4] = (W[4] + p) * un;
}

// (F_n(Wl) - F_n(Wr)) / 2 of the normal Euler flux by the half-difference
// rules, given the half-difference h of the two global-frame states: exact
// to the rounding of the result itself, however close the two states.
__device__ __forceinline__ void normal_flux_half_difference(const float* Wl, const float* Wr, const float* h,
                                                            const float* n, float gm1, float* out) {
    const HDiff<float> rho{Wl[0], Wr[0], h[0]}, E{Wl[4], Wr[4], h[4]};
    const HDiff<float> m[3] = {{Wl[1], Wr[1], h[1]}, {Wl[2], Wr[2], h[2]}, {Wl[3], Wr[3], h[3]}};
    const HDiff<float> mn = hd_add(hd_add(hd_scale(n[0], m[0]), hd_scale(n[1], m[1])), hd_scale(n[2], m[2]));
    const HDiff<float> un = hd_div(mn, rho);
    const HDiff<float> mm = hd_add(hd_add(hd_mul(m[0], m[0]), hd_mul(m[1], m[1])), hd_mul(m[2], m[2]));
    const HDiff<float> p = hd_scale(gm1, hd_add(E, hd_scale(-0.5f, hd_div(mm, rho))));
    out[0] = mn.h;
#pragma unroll
    for (int j = 0; j < 3; ++j) out[1 + j] = hd_mul(m[j], un).h + n[j] * p.h;
    out[4] = hd_mul(hd_add(E, p), un).h;
}

// ------------------------------------------------- FP32 pair numbers --
// A value hi + lo carried as two FP32 numbers (|lo| <= ulp(hi) / 2): about
// 48 significant bits at FP32-pipe speed.  Sums by Knuth's TwoSum, products
// by the FMA form of Dekker's TwoProduct, quotients by one correction of an
// FP32 quotient with the exact residual.  Used where a value of O(|W|) or
// O(|F|) must stay exact to far below FP32 rounding without the FP64 unit
// (the FP32-bulk reference flux).
struct F2 {
    float hi, lo;
};

__device__ __forceinline__ F2 f2_norm(float s, float e) {
    const float h = s + e;
    return {h, e - (h - s)};
}

__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    return f2_norm(s, e);
}

__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e += a.hi * b.lo + a.lo * b.hi;
    return f2_norm(p, e);
}

__device__ __forceinline__ F2 f2_scale(float c, F2 a) {
    const float p = c * a.hi;
    float e = fmaf(c, a.hi, -p);
    e += c * a.lo;
    return f2_norm(p, e);
}

__device__ __forceinline__ F2 f2_div(F2 a, F2 b) {
    const float q = a.hi / b.hi;
    // residual a - q b, exact to the pair's precision
    const F2 qb = f2_mul({q, 0.0f}, b);
    const F2 r = f2_add(a, {-qb.hi, -qb.lo});
    return f2_norm(q, r.hi / b.hi);
}

__device__ __forceinline__ double f2_value(F2 a) { return (double)a.hi + (double)a.lo; }

}  // namespace gks
