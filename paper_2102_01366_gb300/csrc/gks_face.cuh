// gks_face.cuh -- per-Gauss-point pieces of the face flux shared by the flux
// kernels and their adjoint: the reconstruction evaluated at a point, the
// face frame (Eq. rotate-matrix-3d), the rotations into and out of it, and
// the ghost states of boundary faces (Sec. 4.4).
#pragma once

#include "gks_kernels.h"

namespace gks {

// R and its gradient at X (relative to the centroid) from a cell's
// reconstruction record.  FP64 records hold R in centroid-monomial form; FP32
// records hold R minus the cell average and the average's hi / lo parts, and
// val = hi + (R - average).  dev, ahi, alo (FP32, each may be NULL) receive
// R - average at X and the average's parts.
template <typename T>
__device__ __forceinline__ void eval_poly(const T* __restrict__ P, const T* X, T* val, T (*g)[5],
                                          T* dev = nullptr, T* ahi = nullptr, T* alo = nullptr) {
    // the record is 16-byte aligned: load it in vectors
    constexpr int PS = Stride<T>::poly;
    T c[PS];
    if constexpr (sizeof(T) == 4) {
        const float4* p4 = reinterpret_cast<const float4*>(P);
#pragma unroll
        for (int i = 0; i < PS / 4; ++i) {
            const float4 v = __ldg(p4 + i);
            c[4 * i] = v.x;
            c[4 * i + 1] = v.y;
            c[4 * i + 2] = v.z;
            c[4 * i + 3] = v.w;
        }
    } else {
        const double2* p2 = reinterpret_cast<const double2*>(P);
#pragma unroll
        for (int i = 0; i < PS / 2; ++i) {
            const double2 v = __ldg(p2 + i);
            c[2 * i] = v.x;
            c[2 * i + 1] = v.y;
        }
    }
    const T x = X[0], y = X[1], z = X[2];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const T* cq = c + q * 10;
        const T v = cq[0] + cq[1] * x + cq[2] * y + cq[3] * z + cq[4] * x * x + cq[5] * x * y + cq[6] * x * z +
                    cq[7] * y * y + cq[8] * y * z + cq[9] * z * z;
        if constexpr (sizeof(T) == 4) {
            val[q] = c[PHI + q] + v;
            if (dev) dev[q] = v;
            if (ahi) ahi[q] = c[PHI + q];
            if (alo) alo[q] = c[PLO + q];
        } else {
            val[q] = v;
        }
        g[0][q] = cq[1] + T(2) * cq[4] * x + cq[5] * y + cq[6] * z;
        g[1][q] = cq[2] + cq[5] * x + T(2) * cq[7] * y + cq[8] * z;
        g[2][q] = cq[3] + cq[6] * x + cq[8] * y + T(2) * cq[9] * z;
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

// Slip-wall ghost (Sec. 4.4) of a state already in the face frame (x1 along
// the normal): the mirror image across the wall.  rho U1 changes sign; of the
// x1-derivatives all but that of rho U1 change sign; of the x2-, x3-derivatives
// only those of rho U1 do.
template <typename T>
__device__ __forceinline__ void slip_wall_ghost(T* Wt, T (*gt)[5]) {
    Wt[1] = -Wt[1];
    gt[0][0] = -gt[0][0];
    gt[0][2] = -gt[0][2];
    gt[0][3] = -gt[0][3];
    gt[0][4] = -gt[0][4];
    gt[1][1] = -gt[1][1];
    gt[2][1] = -gt[2][1];
}

// Non-slip adiabatic wall at rest (Sec. 4.4) in the face frame: rho and rho E
// kept, the three momenta reversed; every derivative of the momenta kept,
// every derivative of rho and rho E reversed.
template <typename T>
__device__ __forceinline__ void noslip_wall_ghost(T* Wt, T (*gt)[5]) {
    Wt[1] = -Wt[1];
    Wt[2] = -Wt[2];
    Wt[3] = -Wt[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        gt[j][0] = -gt[j][0];
        gt[j][4] = -gt[j][4];
    }
}

// Non-slip isothermal wall at rest (Sec. 4.4) in the face frame, R = 1
// (T = p / rho): the ghost has the interior pressure, the reversed velocity
// and the temperature 2 T_w - T; of the primitive derivatives the velocity's
// and the temperature's are kept and the pressure's reversed, then carried
// back to the conservative derivatives through the chain rule.
template <typename T>
__device__ __forceinline__ void isothermal_wall_ghost(T* Wt, T (*gt)[5], T gm1, T Tw) {
    const T rho = Wt[0], ir = T(1) / rho;
    const T U[3] = {Wt[1] * ir, Wt[2] * ir, Wt[3] * ir};
    const T Q = T(0.5) * (U[0] * U[0] + U[1] * U[1] + U[2] * U[2]);
    const T p = gm1 * (Wt[4] - rho * Q);
    const T Tr = p * ir;
    const T Tl = T(2) * Tw - Tr;
    const T rl = p / Tl;
    Wt[0] = rl;
    Wt[1] = -rl * U[0];
    Wt[2] = -rl * U[1];
    Wt[3] = -rl * U[2];
    Wt[4] = p / gm1 + rl * Q;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T dU[3], dQ = T(0);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            dU[i] = (gt[j][1 + i] - gt[j][0] * U[i]) * ir;
            dQ += U[i] * dU[i];
        }
        const T dp = gm1 * (gt[j][4] - gt[j][0] * Q - rho * dQ);
        const T dT = (dp - gt[j][0] * Tr) * ir;
        // ghost: dU and dT kept, dp reversed; U reversed, so dQ reverses too
        const T dpl = -dp;
        const T drl = (dpl - dT * rl) / Tl;
        gt[j][0] = drl;
#pragma unroll
        for (int i = 0; i < 3; ++i) gt[j][1 + i] = -drl * U[i] + dU[i] * rl;
        gt[j][4] = drl * Q - rl * dQ + dpl / gm1;
    }
}

// a global-frame vector in the face frame (rows of Rm: n, t1, t2)
template <typename T>
__device__ __forceinline__ void rotate_vec(const T (*Rm)[3], const T* v, T* o) {
#pragma unroll
    for (int i = 0; i < 3; ++i) o[i] = Rm[i][0] * v[0] + Rm[i][1] * v[1] + Rm[i][2] * v[2];
}

// Non-slip adiabatic wall moving with velocity Uw (face frame, tangential):
// the ghost's velocity is 2 Uw - U, its density and pressure the interior's;
// of the primitive derivatives the velocity's are kept and the density's and
// pressure's reversed, then carried back to the conservative derivatives.
// At Uw = 0 this is noslip_wall_ghost.
template <typename T>
__device__ __forceinline__ void moving_wall_ghost(T* Wt, T (*gt)[5], T gm1, const T* Uw) {
    const T rho = Wt[0], ir = T(1) / rho;
    const T U[3] = {Wt[1] * ir, Wt[2] * ir, Wt[3] * ir};
    const T Q = T(0.5) * (U[0] * U[0] + U[1] * U[1] + U[2] * U[2]);
    const T p = gm1 * (Wt[4] - rho * Q);
    const T Ul[3] = {T(2) * Uw[0] - U[0], T(2) * Uw[1] - U[1], T(2) * Uw[2] - U[2]};
    const T Ql = T(0.5) * (Ul[0] * Ul[0] + Ul[1] * Ul[1] + Ul[2] * Ul[2]);
    Wt[1] = rho * Ul[0];
    Wt[2] = rho * Ul[1];
    Wt[3] = rho * Ul[2];
    Wt[4] = p / gm1 + rho * Ql;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        T dU[3], dQ = T(0), dQl = T(0);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            dU[i] = (gt[j][1 + i] - gt[j][0] * U[i]) * ir;
            dQ += U[i] * dU[i];
            dQl += Ul[i] * dU[i];
        }
        const T dp = gm1 * (gt[j][4] - gt[j][0] * Q - rho * dQ);
        const T drl = -gt[j][0];
        gt[j][0] = drl;
#pragma unroll
        for (int i = 0; i < 3; ++i) gt[j][1 + i] = drl * Ul[i] + rho * dU[i];
        gt[j][4] = -dp / gm1 + drl * Ql + rho * dQl;
    }
}

// device encoding of a boundary face's missing side (flr): -1 - GKS_BC_*
inline constexpr int FLR_OPEN = -1, FLR_SLIP_WALL = -2, FLR_FIXED = -3, FLR_NOSLIP_WALL = -4,
                     FLR_ISOTHERMAL_WALL = -5, FLR_MOVING_WALL = -6;

// fixed boundary: the interior cell's fixed state (average and gradient)
// extended linearly to the point X (relative to the cell's centroid)
template <typename T>
__device__ __forceinline__ void fixed_ghost(const T* __restrict__ x0, const T* X, T* W, T (*g)[5]) {
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        T v = x0[q];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            g[i][q] = x0[5 + 3 * q + i];
            v += g[i][q] * X[i];
        }
        W[q] = v;
    }
}

}  // namespace gks
