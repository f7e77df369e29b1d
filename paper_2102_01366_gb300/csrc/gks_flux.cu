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

#include "gks_flux.cuh"

namespace gks {

// --------------------------------------------------------------------------
// face flux
// --------------------------------------------------------------------------


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
                eval_poly(poly + c * Stride<T>::poly, X, Wv, g);
            } else if (cell == FLR_FIXED) {
                const int64_t in = side == 0 ? Rc : L;
                const int src = 1 - side;
                const T X[3] = {geo[4 + 9 * src + 3 * k], geo[5 + 9 * src + 3 * k], geo[6 + 9 * src + 3 * k]};
                fixed_ghost(m.fixed + in * Stride<T>::xs, X, Wv, g);
            } else {
                // open boundary: interior cell average, zero gradient
                const int64_t in = side == 0 ? Rc : L;
                for (int q = 0; q < 5; ++q) {
                    Wv[q] = Wavg[in * Stride<T>::xs + q];
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
        // meshes with isothermal or moving walls: the instances that carry
        // their ghosts (gks_flux_xw.cu)
        if (m.xwalls) return launch_flux_xw(m, ph, W, poly, rec, ctrl, dt_override, stage, s, variant, prf);
        auto go = [&](auto kernel) { kernel<<<grid, 2 * FP_GP, 0, s>>>(m, ph, W, poly, rec, ctrl, dt_override); };
        if (variant == 1) {
            if (stage == 1)
                prf ? go(k_flux<T, 40, 3, true, false>) : go(k_flux<T, 40, 3, false, false>);
            else
                prf ? go(k_flux<T, 20, 3, true, false>) : go(k_flux<T, 20, 3, false, false>);
        } else {
            if (stage == 1)
                prf ? go(k_flux<T, 40, 2, true, false>) : go(k_flux<T, 40, 2, false, false>);
            else
                prf ? go(k_flux<T, 20, 2, true, false>) : go(k_flux<T, 20, 2, false, false>);
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
