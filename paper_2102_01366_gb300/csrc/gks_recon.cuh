// gks_recon.cuh -- device pieces of the reconstruction (Sec. 4.1-4.3) and of
// the time-step finalisation, shared by the standalone kernels and the
// persistent stage kernel.
#pragma once

#include <cuda_runtime.h>

#include "gks_cells.cuh"
#include "gks_device.cuh"
#include "gks_kernels.h"

namespace gks {

// ---- bulk copy global -> shared with an mbarrier (sm_90+ async proxy) ----
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one arrival that also announces the bytes the copy will deliver
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// bounded wait for phase `parity`: false if it gave up (each try_wait
// already suspends for a while, so the bound is far beyond any copy time)
constexpr int MBAR_TRIES = 1 << 16;
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    for (int i = 0; i < MBAR_TRIES; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

template <typename T>
struct ReconConst {
    T gm1, eps;
    int weno, order;
};


// The step of every case from its minimum local limit (time-step rule of
// Sec. 5), with dt_fixed and t_end clipping; advances the case times and
// resets the minima for the next update.  One thread per case.
__device__ inline void finalize_cases(unsigned long long* __restrict__ dtmin, double* __restrict__ case_t,
                               double* __restrict__ case_dt, int32_t ncase, double cfl,
                               const double* __restrict__ ctrl) {
    const double dt_fixed = ctrl[CTRL_DT_FIXED], t_end = ctrl[CTRL_T_END];
    for (int k = threadIdx.x; k < ncase; k += blockDim.x) {
        const double mn = __longlong_as_double((long long)dtmin[k]);
        double dt = dt_fixed > 0.0 ? dt_fixed : (mn < INFINITY ? cfl * mn : 0.0);
        double t = case_t[k];
        if (t_end > 0.0) {
            const double rem = t_end - t;
            if (rem <= 1e-12 * t_end) {
                dt = 0.0;
                if (rem > 0.0) t = t_end;
            } else if (dt > rem) {
                dt = rem;
            }
        }
        if (!(dt > 0.0)) dt = 0.0;
        case_dt[k] = dt;
        case_t[k] = t + dt;
        dtmin[k] = (unsigned long long)__double_as_longlong(INFINITY);
    }
}

template <typename T>
struct FinArg {
    unsigned long long* dtmin;
    double* case_t;
    double* case_dt;
    int32_t ncase;
    double cfl;
    const double* ctrl;
};
// Q_a - Q_b of component q of two cell averages: in FP32 bulk from the hi
// and lo parts (exact to the rounding of the difference itself)
template <typename T, typename TO = T>
__device__ __forceinline__ TO avg_diff(const T* __restrict__ X, int64_t a, int64_t b, int q) {
    constexpr int XSR = Stride<T>::xs;
    if constexpr (sizeof(T) == 4)
        return ((TO)X[a * XSR + q] - (TO)X[b * XSR + q]) + ((TO)X[a * XSR + XLO + q] - (TO)X[b * XSR + XLO + q]);
    else
        return X[a * XSR + q] - X[b * XSR + q];
}

// the step-1 operator entry M1[row][c] in the operator precision TO
template <typename T, typename TO>
__device__ __forceinline__ TO m1_at(const DevMesh<T>& m, int row, int64_t c) {
    if constexpr (sizeof(TO) > sizeof(T))
        return m.M1d[row * m.nc + c];
    else
        return m.M1[row * m.nc + c];
}

// The wall-constrained operator slot (Sec. 4.4) of component q of cell c:
// the momenta of a cell with non-slip adiabatic wall faces whose
// constrained stencils were built; NULL otherwise
template <typename T, typename TO, bool WALL = true>
__device__ __forceinline__ const TO* wall_ops(const DevMesh<T>& m, int64_t c, int q) {
    if (!WALL || !m.wslot || q < 1 || q > 3) return nullptr;
    const int32_t w = m.wslot[c];
    if (w < 0) return nullptr;
    if constexpr (sizeof(TO) > sizeof(T))
        return m.wopd + (int64_t)w * WOP_STRIDE;
    else
        return m.wop + (int64_t)w * WOP_STRIDE;
}

// cell average Q0 of component q in TO (FP32 bulk: hi + lo)
template <typename T, typename TO>
__device__ __forceinline__ TO avg_at(const T* __restrict__ X, int64_t c, int q) {
    constexpr int XSR = Stride<T>::xs;
    if constexpr (sizeof(T) == 4)
        return (TO)X[c * XSR + q] + (TO)X[c * XSR + XLO + q];
    else
        return X[c * XSR + q];
}

// P1 slope of cell x for component q (Sec. 4.3, reconstruction step 1):
// b = M1 (Q_nb - Q_x) over the existing neighbours; at a non-slip wall the
// constrained slope b = W1 [Q_nb - Q_x; Q_x] (Sec. 4.4)
template <typename T, typename TO, bool WALL = true>
__device__ __forceinline__ void p1_slope(const DevMesh<T>& m, const T* __restrict__ X, int64_t x, int q, T* b) {
    const int64_t nc = m.nc;
    TO s[3] = {TO(0), TO(0), TO(0)};
    const TO* wo = wall_ops<T, TO, WALL>(m, x, q);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const int nb = m.nbr[f * nc + x];
        if (nb < 0) continue;
        const TO dq = avg_diff<T, TO>(X, nb, x, q);
#pragma unroll
        for (int i = 0; i < 3; ++i) s[i] += (wo ? wo[WOP_W1 + i * 5 + f] : m1_at<T, TO>(m, i * 4 + f, x)) * dq;
    }
    if (wo) {
        const TO q0 = avg_at<T, TO>(X, x, q);
#pragma unroll
        for (int i = 0; i < 3; ++i) s[i] += wo[WOP_W1 + i * 5 + 4] * q0;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) b[i] = (T)s[i];
}

// reconstruction (Sec. 4.1-4.3): the cell's own P1 slopes and, for the
// two-step beta_0, its neighbours' P1 slopes (recomputed here, or read from
// a slopes pass); P2 = M2 d with the block's static data (M2, Gauss points,
// M1, moments) brought into shared memory by one bulk copy that overlaps the
// neighbour gathers;
// smoothness indicators, nonlinear weights, positivity at the cell's 12 face
// Gauss points (Sec. 4.2); R written about the centroid in monomial form.
// TO is the precision of the stencil operators and of their products
// (FP32 bulk: FP32, or FP64 with precision 2; the FP64 path: FP64).
//
// recon_cells: one block of CELLS_PER_BLOCK cells (block index vb) by
// CELL_THREADS threads (tid); sT the block's tile in shared memory and bar
// an initialised mbarrier whose phase `parity` this tile's copy completes
// (thread 0 issues the copy).  The standalone kernel and the persistent
// stage kernel both run it; every thread returns from it (no early exit).
template <typename TO>
using Tile = TO[TILE_ROWS][CELLS_PER_BLOCK];

template <typename T, typename TO, bool WALL>
__device__ __forceinline__ void recon_cells(const DevMesh<T>& m, const ReconConst<T>& rc, const T* __restrict__ X,
                                            const T* __restrict__ slopes_in, T* __restrict__ slopes_out,
                                            T* __restrict__ poly, int32_t* __restrict__ fallback,
                                            int32_t* __restrict__ err, int64_t vb, int tid, Tile<TO>& sT,
                                            unsigned long long* bar, unsigned parity) {
    constexpr unsigned TILE_BYTES = TILE_ROWS * CELLS_PER_BLOCK * sizeof(TO);
    static_assert(TILE_BYTES % 16 == 0, "bulk copies move multiples of 16 bytes");
    const TO* tile = nullptr;
    if constexpr (sizeof(TO) > sizeof(T))
        tile = m.tiled;
    else
        tile = m.tile;
    if (tid == 0) {
        mbar_arrive_expect_tx(bar, TILE_BYTES);
        bulk_load(&sT[0][0], tile + vb * TILE_ROWS * CELLS_PER_BLOCK, TILE_BYTES, bar);
    }
    const int64_t nc = m.nc;
    const CellLane cl = cell_lane(nc, vb, tid);
    const int64_t c = cl.c;
    const int q = cl.q;
    const int lc = (int)(c - vb * CELLS_PER_BLOCK) < CELLS_PER_BLOCK ? (int)(c - vb * CELLS_PER_BLOCK)
                                                                       : CELLS_PER_BLOCK - 1;
    int nb[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) nb[f] = m.nbr[f * nc + c];
    constexpr int XSR = Stride<T>::xs;
    const T Q0 = X[c * XSR + q];
    T Q0lo = T(0);  // lo part of the FP32 pair (FP64: unused)
    if constexpr (sizeof(T) == 4) Q0lo = X[c * XSR + XLO + q];

    // data vector [dQ_f (4); grad Q_{f,l} (12)] of this component
    TO d[16];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const bool ok = nb[f] >= 0;
        const T* xn = X + (ok ? (int64_t)nb[f] : c) * XSR;
        if constexpr (sizeof(T) == 4)
            d[f] = ok ? ((TO)xn[q] - (TO)Q0) + ((TO)xn[XLO + q] - (TO)Q0lo) : TO(0);
        else
            d[f] = ok ? xn[q] - Q0 : T(0);
#pragma unroll
        for (int l = 0; l < 3; ++l) d[4 + 3 * f + l] = ok ? (TO)xn[5 + 3 * q + l] : TO(0);
    }
    // the tile has landed (all threads wait; a give-up is reported, and the
    // values computed from an incomplete tile are never trusted by the host)
    const bool tile_ok = mbar_wait(bar, parity);
    if (!tile_ok && (threadIdx.x & 31) == 0) atomicOr(err, ERR_TIMEOUT);
    // P2 in the zero-mean basis of Eq. base: a = M2 d (at a non-slip wall
    // the momenta's constrained a = W2 [d; Q0], Sec. 4.4)
    const TO* wo = wall_ops<T, TO, WALL>(m, c, q);
    TO q0w = TO(0);
    if (wo) q0w = avg_at<T, TO>(X, c, q);
    T a[9];
    if (wo) {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            TO acc = wo[k * 17 + 16] * q0w;
#pragma unroll
            for (int j = 0; j < 16; ++j) acc += wo[k * 17 + j] * d[j];
            a[k] = (T)acc;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            TO acc = TO(0);
#pragma unroll
            for (int j = 0; j < 16; ++j) acc += sT[TILE_M2 + k * 16 + j][lc] * d[j];
            a[k] = (T)acc;
        }
    }
    const T Mxx = (T)sT[TILE_MOM + 0][lc], Mxy = (T)sT[TILE_MOM + 1][lc], Mxz = (T)sT[TILE_MOM + 2][lc];
    const T Myy = (T)sT[TILE_MOM + 3][lc], Myz = (T)sT[TILE_MOM + 4][lc], Mzz = (T)sT[TILE_MOM + 5][lc];

    const T g22 = T(100.0 / 111.0), g12 = T(10.0 / 111.0), g02 = T(1.0 / 111.0);
    const T g11 = T(10.0 / 11.0), g01 = T(1.0 / 11.0);
    T R[9];
    T b[3] = {T(0), T(0), T(0)};
    if (rc.weno || rc.order == 2) {
        // own P1 slope from the neighbour differences already loaded
        TO bo[3] = {TO(0), TO(0), TO(0)};
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            if (nb[f] < 0) continue;
#pragma unroll
            for (int i = 0; i < 3; ++i) bo[i] += (wo ? wo[WOP_W1 + i * 5 + f] : sT[TILE_M1 + i * 4 + f][lc]) * d[f];
        }
        if (wo) {
#pragma unroll
            for (int i = 0; i < 3; ++i) bo[i] += wo[WOP_W1 + i * 5 + 4] * q0w;
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) b[i] = (T)bo[i];
        if (slopes_out && cl.active) {
#pragma unroll
            for (int i = 0; i < 3; ++i) slopes_out[c * 15 + 3 * q + i] = b[i];
        }
    }
    if (!rc.weno) {
#pragma unroll
        for (int k = 0; k < 9; ++k) R[k] = rc.order == 2 ? (k < 3 ? b[k] : T(0)) : a[k];
    } else {
        const T v23 = (T)sT[TILE_V23][lc], v43 = (T)sT[TILE_V43][lc];
        // smoothness indicators, Eq. smooth-indicator
        const T beta1 = v23 * (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
        // two-step beta_0 from the neighbours' P1 slopes, Eq. p0-non-linear-weight
        T b0j[4];
        int nn = 0;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            if (nb[f] < 0) continue;
            T bj[3];
            if (slopes_in) {
                const T* sj = slopes_in + (int64_t)nb[f] * 15 + 3 * q;
                bj[0] = sj[0];
                bj[1] = sj[1];
                bj[2] = sj[2];
            } else {
                p1_slope<T, TO, WALL>(m, X, nb[f], q, bj);
            }
            b0j[nn++] = v23 * (bj[0] * bj[0] + bj[1] * bj[1] + bj[2] * bj[2]);
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
            const T cl1 = (w1 / (w0 + w1)) / g11;
#pragma unroll
            for (int k = 0; k < 9; ++k) R[k] = k < 3 ? cl1 * b[k] : T(0);
        } else {
            // Hessian rows of P2 and the integrals of its derivatives
            const T H[3][3] = {{T(2) * a[3], a[4], a[5]}, {a[4], T(2) * a[6], a[7]}, {a[5], a[7], T(2) * a[8]}};
            T first = T(0);
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                const T h0 = H[l][0], h1 = H[l][1], h2 = H[l][2];
                const T hMh = h0 * (Mxx * h0 + Mxy * h1 + Mxz * h2) + h1 * (Mxy * h0 + Myy * h1 + Myz * h2) +
                              h2 * (Mxz * h0 + Myz * h1 + Mzz * h2);
                first += a[l] * a[l] + hMh;
            }
            const T second = H[0][0] * H[0][0] + a[4] * a[4] + a[5] * a[5] + H[1][1] * H[1][1] + a[7] * a[7] +
                             H[2][2] * H[2][2];
            const T beta2 = v23 * first + v43 * second;
            // global smoothness indicator and nonlinear weights, Eq. non-linear-weight
            const T sigma = pow43(T(0.5) * (d_abs(beta2 - beta1) + d_abs(beta2 - beta0)));
            const T r0 = sigma / (rc.eps + beta0), r1 = sigma / (rc.eps + beta1), r2 = sigma / (rc.eps + beta2);
            const T w0 = g02 * (T(1) + r0 * r0), w1 = g12 * (T(1) + r1 * r1), w2 = g22 * (T(1) + r2 * r2);
            const T iw = T(1) / (w0 + w1 + w2);
            const T c2 = (w2 * iw) / g22;
            const T cb = (w1 * iw) / g11 - c2 * g12 / g11;
#pragma unroll
            for (int k = 0; k < 9; ++k) R[k] = c2 * a[k] + (k < 3 ? cb * b[k] : T(0));
        }
    }
    // constant of the monomial form, less the cell average: R(centroid) - Q0
    const T dc = (T)(-((TO)R[3] * sT[TILE_MOM + 0][lc] + (TO)R[4] * sT[TILE_MOM + 1][lc] +
                       (TO)R[5] * sT[TILE_MOM + 2][lc] + (TO)R[6] * sT[TILE_MOM + 3][lc] +
                       (TO)R[7] * sT[TILE_MOM + 4][lc] + (TO)R[8] * sT[TILE_MOM + 5][lc]));
    const T c0 = Q0 + dc;
    // positivity: the 5 lanes of the cell exchange their values at each point
    bool bad = false;
#pragma unroll 4
    for (int g = 0; g < 12; ++g) {
        const T gx = (T)sT[TILE_G + g * 3 + 0][lc];
        const T gy = (T)sT[TILE_G + g * 3 + 1][lc];
        const T gz = (T)sT[TILE_G + g * 3 + 2][lc];
        const T v = c0 + R[0] * gx + R[1] * gy + R[2] * gz + R[3] * gx * gx + R[4] * gx * gy + R[5] * gx * gz +
                    R[6] * gy * gy + R[7] * gy * gz + R[8] * gz * gz;
        const T rho = __shfl_sync(0xffffffffu, v, cl.base + 0);
        const T m1 = __shfl_sync(0xffffffffu, v, cl.base + 1);
        const T m2 = __shfl_sync(0xffffffffu, v, cl.base + 2);
        const T m3 = __shfl_sync(0xffffffffu, v, cl.base + 3);
        const T en = __shfl_sync(0xffffffffu, v, cl.base + 4);
        const T pr = rc.gm1 * (en - T(0.5) * (m1 * m1 + m2 * m2 + m3 * m3) / rho);
        if (!(rho > T(0)) || !(pr > T(0))) bad = true;
    }
    if (!tile_ok) mbar_wait(bar, parity);  // a late copy lands before the block exits
    if (cl.active) {
        T* rec = poly + c * Stride<T>::poly;
        T* out = rec + q * 10;
        if constexpr (sizeof(T) == 4) {
            // FP32: R(centroid) - Q0 and the average's hi / lo parts
            out[0] = bad ? T(0) : dc;
            rec[PHI + q] = Q0;
            rec[PLO + q] = Q0lo;
        } else {
            out[0] = bad ? Q0 : c0;
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) out[1 + k] = bad ? T(0) : R[k];
        if (fallback && q == 0) fallback[c] = bad ? 1 : 0;
    }
}

}  // namespace gks
