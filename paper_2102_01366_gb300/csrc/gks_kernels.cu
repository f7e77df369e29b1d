// gks_kernels.cu -- sm_103a kernels of one two-stage step of the compact
// gas-kinetic scheme on tetrahedra (FP64 and FP32-bulk instantiations).
//
//   k_slopes   reconstruction step 1: P1 slopes per cell (Sec. 4.3)
//   k_recon    reconstruction step 2: P2 by the 9x16 operator, smoothness
//              indicators, two-step beta_0, nonlinear weights, positivity
//              (Sec. 4.1-4.3); R written about the centroid in monomial form
//   k_flux     face-ordered: R of both cells at the 3 Gauss points, face
//              frame, kinetic solution (Sec. 2.2, 4.5), weighted face record
//              of the stage (Sec. 3 Eqs. linear-system, s2o4, step-du)
//   k_update1  cell-ordered gather of the 4 face records (CSR, signed):
//              W*, grad W* and the saved stage-1 terms
//   k_update2  W^{n+1}, grad W^{n+1}; per-block time-step minimum and
//              residual sums for the next step
//   k_dt_*     time-step rule of Sec. 5 (two-pass deterministic minimum)
//
// No atomics on data: every sum has a fixed order, so results are
// reproducible run to run.
#include <cuda_runtime.h>

#include "gks_device.cuh"
#include "gks_kernels.h"

namespace gks {

template <typename T>
struct ReconConst {
    T gm1, eps;
    int weno, order;
};

// --------------------------------------------------------------------------
// reconstruction step 1
// --------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(CELL_THREADS) k_slopes(DevMesh<T> m, const T* __restrict__ W,
                                                          T* __restrict__ slopes) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m.nc) return;
    const int64_t nc = m.nc;
    T Q0[5], b[5][3];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        Q0[q] = W[q * nc + c];
        b[q][0] = b[q][1] = b[q][2] = T(0);
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const int nb = m.nbr[f * nc + c];
        if (nb < 0) continue;
        const T m0 = m.M1[(0 * 4 + f) * nc + c];
        const T m1 = m.M1[(1 * 4 + f) * nc + c];
        const T m2 = m.M1[(2 * 4 + f) * nc + c];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const T dq = W[q * nc + nb] - Q0[q];
            b[q][0] += m0 * dq;
            b[q][1] += m1 * dq;
            b[q][2] += m2 * dq;
        }
    }
    T* out = slopes + c * 15;
#pragma unroll
    for (int q = 0; q < 5; ++q)
#pragma unroll
        for (int i = 0; i < 3; ++i) out[q * 3 + i] = b[q][i];
}

// --------------------------------------------------------------------------
// reconstruction step 2
// --------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(CELL_THREADS) k_recon(DevMesh<T> m, ReconConst<T> rc,
                                                         const T* __restrict__ W,
                                                         const T* __restrict__ dW,
                                                         const T* __restrict__ slopes,
                                                         T* __restrict__ poly,
                                                         int32_t* __restrict__ fallback) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m.nc) return;
    const int64_t nc = m.nc;
    int nb[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) nb[f] = m.nbr[f * nc + c];
    T Q0[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) Q0[q] = W[q * nc + c];

    // data vectors [dQ_f (4); grad Q_{f,l} (12)] of all components
    T d[5][16];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const bool ok = nb[f] >= 0;
        const int64_t n = ok ? nb[f] : c;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            d[q][f] = ok ? W[q * nc + n] - Q0[q] : T(0);
#pragma unroll
            for (int l = 0; l < 3; ++l) d[q][4 + 3 * f + l] = ok ? dW[(3 * q + l) * nc + n] : T(0);
        }
    }
    // P2 in the zero-mean basis: a = M2 d  (M2 streamed once, SoA, coalesced)
    T a[5][9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
#pragma unroll
        for (int q = 0; q < 5; ++q) a[q][k] = T(0);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const T mk = m.M2[(k * 16 + j) * nc + c];
#pragma unroll
            for (int q = 0; q < 5; ++q) a[q][k] += mk * d[q][j];
        }
    }
    T Mxx = m.mom2[0 * nc + c], Mxy = m.mom2[1 * nc + c], Mxz = m.mom2[2 * nc + c];
    T Myy = m.mom2[3 * nc + c], Myz = m.mom2[4 * nc + c], Mzz = m.mom2[5 * nc + c];

    // final R coefficients (basis form; the constant is Q0)
    T R[5][9];
    const bool need_b = rc.weno || rc.order == 2;
    const T g22 = T(100.0 / 111.0), g12 = T(10.0 / 111.0), g02 = T(1.0 / 111.0);
    const T g11 = T(10.0 / 11.0), g01 = T(1.0 / 11.0);
    const T v23 = m.vol23[c], v43 = m.vol43[c];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        T b[3] = {T(0), T(0), T(0)};
        if (need_b) {
#pragma unroll
            for (int i = 0; i < 3; ++i) b[i] = slopes[c * 15 + 3 * q + i];
        }
        if (!rc.weno) {
            if (rc.order == 2) {
#pragma unroll
                for (int k = 0; k < 9; ++k) R[q][k] = k < 3 ? b[k] : T(0);
            } else {
#pragma unroll
                for (int k = 0; k < 9; ++k) R[q][k] = a[q][k];
            }
            continue;
        }
        // smoothness indicators, Eq. smooth-indicator
        const T beta1 = v23 * (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
        // two-step beta_0 from the neighbours' step-1 slopes, Eq. p0-non-linear-weight
        T b0j[4];
        int nn = 0;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            if (nb[f] < 0) continue;
            const T* s = slopes + (int64_t)nb[f] * 15 + 3 * q;
            const T x = s[0], y = s[1], z = s[2];
            b0j[nn++] = v23 * (x * x + y * y + z * z);
        }
        T beta0 = T(0);
        if (nn > 0) {
            T sum = T(0);
            int npair = 0;
            for (int j = 0; j < nn; ++j)
                for (int k = 0; k < j; ++k) {
                    sum += d_abs(b0j[j] - b0j[k]);
                    ++npair;
                }
            const T s1 = npair ? pow43(sum / T(npair)) : T(0);
            T ws = T(0), acc = T(0);
            for (int j = 0; j < nn; ++j) {
                const T w1 = T(1) + s1 / (rc.eps + b0j[j]);
                ws += w1;
                acc += w1 * b0j[j];
            }
            beta0 = acc / ws;
        }
        if (rc.order == 2) {
            const T sigma = pow43(d_abs(beta1 - beta0));
            const T r0 = sigma / (rc.eps + beta0), r1 = sigma / (rc.eps + beta1);
            const T w0 = g01 * (T(1) + r0 * r0), w1 = g11 * (T(1) + r1 * r1);
            const T cl = (w1 / (w0 + w1)) / g11;
#pragma unroll
            for (int k = 0; k < 9; ++k) R[q][k] = k < 3 ? cl * b[k] : T(0);
            continue;
        }
        const T* aq = a[q];
        // Hessian rows of P2 and the integrals of its derivatives
        const T H[3][3] = {{T(2) * aq[3], aq[4], aq[5]},
                           {aq[4], T(2) * aq[6], aq[7]},
                           {aq[5], aq[7], T(2) * aq[8]}};
        T first = T(0);
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const T h0 = H[l][0], h1 = H[l][1], h2 = H[l][2];
            const T hMh = h0 * (Mxx * h0 + Mxy * h1 + Mxz * h2) + h1 * (Mxy * h0 + Myy * h1 + Myz * h2) +
                          h2 * (Mxz * h0 + Myz * h1 + Mzz * h2);
            first += aq[l] * aq[l] + hMh;
        }
        const T second = H[0][0] * H[0][0] + aq[4] * aq[4] + aq[5] * aq[5] + H[1][1] * H[1][1] +
                         aq[7] * aq[7] + H[2][2] * H[2][2];
        const T beta2 = v23 * first + v43 * second;
        // global smoothness indicator and nonlinear weights, Eq. non-linear-weight
        const T sigma = pow43(T(0.5) * (d_abs(beta2 - beta1) + d_abs(beta2 - beta0)));
        const T r0 = sigma / (rc.eps + beta0), r1 = sigma / (rc.eps + beta1),
                r2 = sigma / (rc.eps + beta2);
        const T w0 = g02 * (T(1) + r0 * r0), w1 = g12 * (T(1) + r1 * r1), w2 = g22 * (T(1) + r2 * r2);
        const T iw = T(1) / (w0 + w1 + w2);
        const T c2 = (w2 * iw) / g22;
        const T cb = (w1 * iw) / g11 - c2 * g12 / g11;
#pragma unroll
        for (int k = 0; k < 9; ++k) R[q][k] = c2 * aq[k] + (k < 3 ? cb * b[k] : T(0));
    }

    // constant term of the monomial form, then the positivity check at the
    // 12 Gauss points of the cell's faces (Sec. 4.2)
    T c0[5];
#pragma unroll
    for (int q = 0; q < 5; ++q)
        c0[q] = Q0[q] - (R[q][3] * Mxx + R[q][4] * Mxy + R[q][5] * Mxz + R[q][6] * Myy +
                         R[q][7] * Myz + R[q][8] * Mzz);
    bool bad = false;
#pragma unroll 1
    for (int g = 0; g < 12; ++g) {
        const T X = m.cgp[(g * 3 + 0) * nc + c];
        const T Y = m.cgp[(g * 3 + 1) * nc + c];
        const T Z = m.cgp[(g * 3 + 2) * nc + c];
        T v[5];
#pragma unroll
        for (int q = 0; q < 5; ++q)
            v[q] = c0[q] + R[q][0] * X + R[q][1] * Y + R[q][2] * Z + R[q][3] * X * X + R[q][4] * X * Y +
                   R[q][5] * X * Z + R[q][6] * Y * Y + R[q][7] * Y * Z + R[q][8] * Z * Z;
        const T pr = rc.gm1 * (v[4] - T(0.5) * (v[1] * v[1] + v[2] * v[2] + v[3] * v[3]) / v[0]);
        if (!(v[0] > T(0)) || !(pr > T(0))) bad = true;
    }
    T* out = poly + c * 50;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        out[q * 10] = bad ? Q0[q] : c0[q];
#pragma unroll
        for (int k = 0; k < 9; ++k) out[q * 10 + 1 + k] = bad ? T(0) : R[q][k];
    }
    if (fallback) fallback[c] = bad ? 1 : 0;
}

// --------------------------------------------------------------------------
// face flux
// --------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void eval_poly(const T* __restrict__ P, const T* X, T* val, T (*g)[5]) {
    const T x = X[0], y = X[1], z = X[2];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const T* c = P + q * 10;
        val[q] = c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * x + c[5] * x * y + c[6] * x * z +
                 c[7] * y * y + c[8] * y * z + c[9] * z * z;
        g[0][q] = c[1] + T(2) * c[4] * x + c[5] * y + c[6] * z;
        g[1][q] = c[2] + c[5] * x + T(2) * c[7] * y + c[8] * z;
        g[2][q] = c[3] + c[6] * x + c[8] * y + T(2) * c[9] * z;
    }
}

// rows of the face frame: n, t1, t2 (Eq. rotate-matrix-3d; n1 = -1 uses the
// reflection diag(-1, -1, 1) of the velocity block)
template <typename T>
__device__ __forceinline__ void face_frame(const T* n, T (*Rm)[3]) {
    const T n1 = n[0], n2 = n[1], n3 = n[2];
    Rm[0][0] = n1;
    Rm[0][1] = n2;
    Rm[0][2] = n3;
    if (n1 == T(-1)) {
        Rm[1][0] = T(0); Rm[1][1] = T(-1); Rm[1][2] = T(0);
        Rm[2][0] = T(0); Rm[2][1] = T(0); Rm[2][2] = T(1);
        return;
    }
    const T r = T(1) / (T(1) + n1);
    Rm[1][0] = -n2;
    Rm[1][1] = n1 + n3 * n3 * r;
    Rm[1][2] = -n2 * n3 * r;
    Rm[2][0] = -n3;
    Rm[2][1] = -n2 * n3 * r;
    Rm[2][2] = T(1) - n3 * n3 * r;
}

template <typename T>
__device__ __forceinline__ void to_local(const T (*Rm)[3], const T* W, const T (*g)[5], T* Wt,
                                         T (*gt)[5]) {
    Wt[0] = W[0];
    Wt[4] = W[4];
#pragma unroll
    for (int j = 0; j < 3; ++j) Wt[1 + j] = Rm[j][0] * W[1] + Rm[j][1] * W[2] + Rm[j][2] * W[3];
    // directions first: h_j = sum_i R_ji g_i, then the momentum components
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T h[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) h[q] = Rm[j][0] * g[0][q] + Rm[j][1] * g[1][q] + Rm[j][2] * g[2][q];
        gt[j][0] = h[0];
        gt[j][4] = h[4];
#pragma unroll
        for (int k = 0; k < 3; ++k) gt[j][1 + k] = Rm[k][0] * h[1] + Rm[k][1] * h[2] + Rm[k][2] * h[3];
    }
}

template <typename T>
__device__ __forceinline__ void to_global(const T (*Rm)[3], T* v) {
    const T a = v[1], b = v[2], c = v[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) v[1 + i] = Rm[0][i] * a + Rm[1][i] * b + Rm[2][i] * c;
}

template <typename T, int NR>
__global__ void __launch_bounds__(3 * FLUX_FACES) k_flux(DevMesh<T> m, Phys<T> ph,
                                                          const T* __restrict__ Wavg,
                                                          const T* __restrict__ poly,
                                                          T* __restrict__ rec,
                                                          const double* __restrict__ ctrl,
                                                          double dt_override) {
    __shared__ T red[FLUX_FACES * 3 * NR];
    const double dtd = dt_override > 0.0 ? dt_override : ctrl[CTRL_DT];
    if (!(dtd > 0.0)) return;  // no-op step (grid-uniform)
    const T dt = (T)dtd;
    const int lf = threadIdx.x / 3;
    const int k = threadIdx.x - 3 * lf;
    const int64_t f = (int64_t)blockIdx.x * FLUX_FACES + lf;
    T* mine = red + (lf * 3 + k) * NR;
    if (f < m.nf) {
        const int L = m.flr[f], Rc = m.flr[m.nf + f];
        const T* geo = m.fgeo + f * FGEO;
        const T n[3] = {geo[0], geo[1], geo[2]};
        const T w = geo[3];
        T WL[5], gL[3][5], WR[5], gR[3][5];
        if (L >= 0) {
            const T X[3] = {geo[4 + 3 * k], geo[5 + 3 * k], geo[6 + 3 * k]};
            eval_poly(poly + (int64_t)L * 50, X, WL, gL);
        }
        if (Rc >= 0) {
            const T X[3] = {geo[13 + 3 * k], geo[14 + 3 * k], geo[15 + 3 * k]};
            eval_poly(poly + (int64_t)Rc * 50, X, WR, gR);
        }
        // open boundary: the missing side is the interior cell's average with
        // zero gradient (zeroth-order extrapolation; the paper leaves outflow
        // boundaries open, and copying the interior Gauss-point state is not
        // stable)
        if (L < 0 || Rc < 0) {
            const int64_t in = L < 0 ? Rc : L;
            T* Wg = L < 0 ? WL : WR;
            T (*gg)[5] = L < 0 ? gL : gR;
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                Wg[q] = Wavg[q * m.nc + in];
                gg[0][q] = gg[1][q] = gg[2][q] = T(0);
            }
        }
        T Rm[3][3];
        face_frame(n, Rm);
        T tWL[5], tgL[3][5], tWR[5], tgR[3][5];
        to_local(Rm, WL, gL, tWL, tgL);
        to_local(Rm, WR, gR, tWR, tgR);
        T Fh[5], D[5], W0[5], dWt[5];
        gks_point(ph, tWL, tgL, tWR, tgR, dt, Fh, D, W0, dWt);
        to_global(Rm, Fh);
        to_global(Rm, D);
        to_global(Rm, W0);
        to_global(Rm, dWt);
        if (NR == 40) {
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                // dt L + dt^2/6 L_t = 8/3 Fh - 1/3 F = 2 Fh - D / 3 (Eqs. linear-system, s2o4)
                mine[q] = w * Fh[q];
                mine[5 + q] = w * (T(2) * Fh[q] - D[q] * T(1.0 / 3.0));
                const T ws = w * (W0[q] + T(0.5) * dWt[q]);  // f* = f^n + dt/2 f_t^n
                const T w0 = w * W0[q];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    mine[10 + 3 * q + i] = ws * n[i];
                    mine[25 + 3 * q + i] = w0 * n[i];
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                // dt^2/3 L_t(W*) = 4/3 (F* - 2 Fh*)
                mine[q] = w * T(4.0 / 3.0) * D[q];
                const T dg = w * dWt[q];  // f^{n+1} = f^n + dt f_t^*
#pragma unroll
                for (int i = 0; i < 3; ++i) mine[5 + 3 * q + i] = dg * n[i];
            }
        }
    }
    __syncthreads();
    // sum the three Gauss points of each face; coalesced record store
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
// cell updates
// --------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(CELL_THREADS) k_update1(DevMesh<T> m, DevState<T> st) {
    const double dtd = st.ctrl[CTRL_DT];
    if (!(dtd > 0.0)) return;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m.nc) return;
    const int64_t nc = m.nc;
    CSum<T> fh[5], s1[5];
    T gs[15], g0[15];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        fh[q].init();
        s1[q].init();
    }
#pragma unroll
    for (int j = 0; j < 15; ++j) gs[j] = g0[j] = T(0);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const int e = m.cface[f * nc + c];
        const T s = (e & 1) ? T(-1) : T(1);
        const T* r = st.rec + (int64_t)(e >> 1) * 40;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            fh[q].add(s * r[q]);
            s1[q].add(s * r[5 + q]);
        }
#pragma unroll
        for (int j = 0; j < 15; ++j) {
            gs[j] += s * r[10 + j];
            g0[j] += s * r[25 + j];
        }
    }
    const double iv = m.inv_vol[c];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        // W* = W^n - (1/|Omega|) sum s sum_k w Fh  (Eq. s2o4, first stage)
        st.Ws[q * nc + c] = (T)(st.Wd[q * nc + c] - fh[q].value() * iv);
        st.S[q * nc + c] = s1[q].value();
    }
    const T ivr = (T)iv;
#pragma unroll
    for (int j = 0; j < 15; ++j) {
        st.dWs[j * nc + c] = gs[j] * ivr;  // Eq. gauss-formula at t* (Eq. step-du)
        st.G[j * nc + c] = g0[j];
    }
}

// deterministic block reduction of one min and five sums
__device__ __forceinline__ void block_reduce_part(double mn, const double* sums, double* out) {
    __shared__ double smin[CELL_THREADS];
    __shared__ double ssum[5][CELL_THREADS];
    const int t = threadIdx.x;
    smin[t] = mn;
#pragma unroll
    for (int q = 0; q < 5; ++q) ssum[q][t] = sums[q];
    __syncthreads();
    for (int s = CELL_THREADS / 2; s > 0; s >>= 1) {
        if (t < s) {
            smin[t] = fmin(smin[t], smin[t + s]);
#pragma unroll
            for (int q = 0; q < 5; ++q) ssum[q][t] += ssum[q][t + s];
        }
        __syncthreads();
    }
    if (t == 0) {
        out[PART_DTMIN] = smin[0];
#pragma unroll
        for (int q = 0; q < 5; ++q) out[PART_RES + q] = ssum[q][0];
    }
}

template <typename T>
__global__ void __launch_bounds__(CELL_THREADS) k_update2(DevMesh<T> m, HostPhys p, DevState<T> st) {
    const double dtd = st.ctrl[CTRL_DT];
    if (!(dtd > 0.0)) return;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nc = m.nc;
    double mn = INFINITY;
    double res[5] = {0, 0, 0, 0, 0};
    if (c < nc) {
        CSum<T> f2[5];
        T dg[15];
#pragma unroll
        for (int q = 0; q < 5; ++q) f2[q].init();
#pragma unroll
        for (int j = 0; j < 15; ++j) dg[j] = T(0);
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const int e = m.cface[f * nc + c];
            const T s = (e & 1) ? T(-1) : T(1);
            const T* r = st.rec + (int64_t)(e >> 1) * 20;
#pragma unroll
            for (int q = 0; q < 5; ++q) f2[q].add(s * r[q]);
#pragma unroll
            for (int j = 0; j < 15; ++j) dg[j] += s * r[5 + j];
        }
        const double iv = m.inv_vol[c];
        T Wn[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            // W^{n+1} |Omega| = W^n |Omega| - [dt F + dt^2/6 F_t](W^n)
            //                   - [dt^2/3 F_t](W*)   (Eq. s2o4, second stage)
            const double inc = ((st.S[q * nc + c] + (double)f2[q].hi) + (double)f2[q].lo) * iv;
            const double wn = st.Wd[q * nc + c] - inc;
            st.Wd[q * nc + c] = wn;
            Wn[q] = (T)wn;
            if ((void*)st.Wr != (void*)st.Wd) st.Wr[q * nc + c] = Wn[q];
            const double r = inc / dtd;
            res[q] = r * r;
        }
        const T ivr = (T)iv;
#pragma unroll
        for (int j = 0; j < 15; ++j) st.dW[j * nc + c] = (st.G[j * nc + c] + dg[j]) * ivr;
        const double pr = (p.gamma - 1.0) * ((double)Wn[4] - 0.5 * ((double)Wn[1] * Wn[1] + (double)Wn[2] * Wn[2] +
                                                                    (double)Wn[3] * Wn[3]) / (double)Wn[0]);
        if (!(Wn[0] > T(0)) || !(pr > 0.0)) atomicOr(st.err, ERR_STATE);
        else mn = local_dt(Wn, m.dr[c], p);
    }
    block_reduce_part(mn, res, st.part + (int64_t)blockIdx.x * PART_N);
    if (blockIdx.x == 0 && threadIdx.x == 0) st.ctrl[CTRL_T] += dtd;
}

template <typename T>
__global__ void __launch_bounds__(CELL_THREADS) k_dt_partials(DevMesh<T> m, HostPhys p,
                                                               const T* __restrict__ W,
                                                               double* __restrict__ part) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double mn = INFINITY;
    double zero[5] = {0, 0, 0, 0, 0};
    if (c < m.nc) {
        T Wv[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) Wv[q] = W[q * m.nc + c];
        mn = local_dt(Wv, m.dr[c], p);
    }
    block_reduce_part(mn, zero, part + (int64_t)blockIdx.x * PART_N);
}

__global__ void k_dt_finalize(const double* __restrict__ part, int nblk, double cfl,
                              double* __restrict__ ctrl) {
    __shared__ double smin[256];
    double mn = INFINITY;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) mn = fmin(mn, part[(int64_t)b * PART_N]);
    smin[threadIdx.x] = mn;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double dt = ctrl[CTRL_DT_FIXED] > 0.0 ? ctrl[CTRL_DT_FIXED] : cfl * smin[0];
        const double t_end = ctrl[CTRL_T_END];
        if (t_end > 0.0) {
            const double rem = t_end - ctrl[CTRL_T];
            if (rem <= 1e-12 * t_end) {
                dt = 0.0;
                if (rem > 0.0) ctrl[CTRL_T] = t_end;
            } else if (dt > rem) {
                dt = rem;
            }
        }
        if (!(dt > 0.0)) dt = 0.0;
        ctrl[CTRL_DT] = dt;
    }
}

__global__ void k_set_control(double* ctrl, double dt_fixed, double t_end, int reset) {
    if (threadIdx.x == 0) {
        ctrl[CTRL_DT_FIXED] = dt_fixed;
        ctrl[CTRL_T_END] = t_end;
        if (reset) {
            ctrl[CTRL_T] = 0.0;
            ctrl[CTRL_DT] = 0.0;
        }
    }
}

template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ in, B* __restrict__ out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (B)in[i];
}

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------
static inline unsigned cell_grid(int64_t nc) { return (unsigned)((nc + CELL_THREADS - 1) / CELL_THREADS); }

int update_blocks(int64_t nc) { return (int)cell_grid(nc); }

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
    return ph;
}

template <typename T>
cudaError_t Launch<T>::slopes(const DevMesh<T>& m, const T* W, T* slopes, cudaStream_t s) {
    if (m.nc == 0) return cudaSuccess;
    k_slopes<T><<<cell_grid(m.nc), CELL_THREADS, 0, s>>>(m, W, slopes);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::recon(const DevMesh<T>& m, const HostPhys& p, const T* W, const T* dW,
                             const T* slopes, T* poly, int32_t* fallback, cudaStream_t s) {
    if (m.nc == 0) return cudaSuccess;
    ReconConst<T> rc;
    rc.gm1 = (T)(p.gamma - 1.0);
    rc.eps = (T)p.eps_weno;
    rc.weno = p.weno;
    rc.order = p.order;
    k_recon<T><<<cell_grid(m.nc), CELL_THREADS, 0, s>>>(m, rc, W, dW, slopes, poly, fallback);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::flux(const DevMesh<T>& m, const HostPhys& p, const T* W, const T* poly, T* rec,
                            const double* ctrl, double dt_override, int stage, cudaStream_t s) {
    if (m.nf == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((m.nf + FLUX_FACES - 1) / FLUX_FACES);
    const Phys<T> ph = make_phys<T>(p);
    if (stage == 1)
        k_flux<T, 40><<<grid, 3 * FLUX_FACES, 0, s>>>(m, ph, W, poly, rec, ctrl, dt_override);
    else
        k_flux<T, 20><<<grid, 3 * FLUX_FACES, 0, s>>>(m, ph, W, poly, rec, ctrl, dt_override);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::update1(const DevMesh<T>& m, const DevState<T>& st, cudaStream_t s) {
    if (m.nc == 0) return cudaSuccess;
    k_update1<T><<<cell_grid(m.nc), CELL_THREADS, 0, s>>>(m, st);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::update2(const DevMesh<T>& m, const HostPhys& p, const DevState<T>& st,
                               cudaStream_t s) {
    if (m.nc == 0) return cudaSuccess;
    k_update2<T><<<cell_grid(m.nc), CELL_THREADS, 0, s>>>(m, p, st);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::dt_partials(const DevMesh<T>& m, const HostPhys& p, const T* W,
                                   double* part, cudaStream_t s) {
    if (m.nc == 0) return cudaSuccess;
    k_dt_partials<T><<<cell_grid(m.nc), CELL_THREADS, 0, s>>>(m, p, W, part);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::to_double(const T* in, double* out, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_convert<T, double><<<(unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Launch<T>::from_double(const double* in, T* out, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_convert<double, T><<<(unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_dt_finalize(const double* part, int nblk, double cfl, double* ctrl, cudaStream_t s) {
    k_dt_finalize<<<1, 256, 0, s>>>(part, nblk, cfl, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_set_control(double* ctrl, double dt_fixed, double t_end, int reset_time,
                               cudaStream_t s) {
    k_set_control<<<1, 32, 0, s>>>(ctrl, dt_fixed, t_end, reset_time);
    return cudaGetLastError();
}

template struct Launch<double>;
template struct Launch<float>;

}  // namespace gks
