// gks_kernels.h -- device data views and kernel launchers of libgks.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace gks {

// control block in device memory (doubles)
enum { CTRL_T = 0, CTRL_DT = 1, CTRL_DT_FIXED = 2, CTRL_T_END = 3, CTRL_N = 8 };
// per-block partial results of the update / time-step kernels
enum { PART_DTMIN = 0, PART_RES = 1, PART_N = 6 };
// device error flags
enum { ERR_STATE = 1, ERR_TIMEOUT = 2 };

constexpr int FLUX_FACES = 32;       // faces per flux block (3 threads each)
constexpr int CELL_THREADS = 128;    // threads per cell-kernel block
constexpr int CELLS_PER_BLOCK = 24;  // 4 warps x 6 cells, 5 lanes per cell
constexpr int FGEO = 24;             // reals per face geometry record
constexpr int POLY_STRIDE = 52;      // reals per cell reconstruction record, FP64 (50 used)
constexpr int XS = 20;               // reals per cell working-state record, FP64: W (5), grad W (15, 3q+i)
// FP32 bulk keeps each cell average as an unevaluated pair hi + lo of FP32
// numbers (the FP64 average to ~48 bits), so that differences between
// neighbouring averages stay exact to FP32 rounding of the difference:
//   working state [nc][28]: W hi (5), grad W (15), W lo (5), pad (3)
//   reconstruction record [nc][60]: per component the constant R(centroid)
//   minus the average and the 9 slopes/curvatures (50), the average's hi (5)
//   and lo (5) parts
constexpr int XS32 = 28;
// FP32 stage-1 face records: the 40 entries of the definition (the flux and
// interface-state entries relative to the mean W_m of the face's two cell
// averages), then the reference flux (dt / 2) A F_n(W_m) as FP32 hi (5) and
// lo (5) parts
constexpr int REC1_F32 = 50, REC1_REF = 40;
constexpr int XLO = 20;              // offset of the lo parts in an FP32 working-state record
constexpr int POLY_STRIDE32 = 60;
constexpr int PHI = 50, PLO = 55;    // offsets of the average's hi / lo parts in an FP32 record
template <typename T>
struct Stride {
    static constexpr int xs = sizeof(T) == 4 ? XS32 : XS;
    static constexpr int poly = sizeof(T) == 4 ? POLY_STRIDE32 : POLY_STRIDE;
};
// Per-block tile of the reconstruction's static cell data, one contiguous
// [TILE_ROWS][CELLS_PER_BLOCK] record per block of cells, loaded into shared
// memory by one bulk copy: M2 (144 rows), the cell's 12 face Gauss points
// about its centroid (36), M1 (12), central second moments (6), |Omega|^(2/3),
// |Omega|^(4/3).
enum { TILE_M2 = 0, TILE_G = 144, TILE_M1 = 180, TILE_MOM = 192, TILE_V23 = 198, TILE_V43 = 199, TILE_ROWS = 200 };
// a wall-constrained operator slot: W2 [9][17] (P2 from [data (16); Q0])
// then W1 [3][5] (P1 slopes from [dQ_f (4); Q0])
enum { WOP_W1 = 153, WOP_STRIDE = 168 };

template <typename T>
struct DevMesh {
    int64_t nc, nf;
    int32_t ncase;
    const int32_t* cell_case;  // [nc] case of each cell (ascending)
    const int32_t* nbr;    // [4][nc], -1 = none
    const int32_t* cface;  // [4][nc] face * 2 + side (side 1 = right)
    const double* inv_vol; // [nc]
    const T* dr;           // [nc]
    const T* M1;           // [12][nc]
    const T* tile;         // [blocks][TILE_ROWS][CELLS_PER_BLOCK] reconstruction data
    // FP32 bulk with FP64 stencil operators (precision 2): the same two in
    // FP64, M1 and tile NULL (else these are NULL)
    const double* M1d;
    const double* tiled;
    const int32_t* flr;    // [2][nf]
    const T* fgeo;         // [nf][FGEO]: n(3), w, XL(9), XR(9), pad
    const float* fan;      // FP32 bulk: [nf][6] face area vectors A n as FP32 hi / lo pairs (NULL in FP64)
    const T* fixed;        // [nc][Stride<T>::xs] state held by fixed boundary faces (NULL: none)
    // Sec. 4.4 wall-constrained momentum stencils (NULL: none): slot of each
    // cell (-1: none) and per slot W2 [9][17] at 0, W1 [3][5] at WOP_W1, in
    // the operator precision (wop; precision 2: wopd)
    const int32_t* wslot;
    const T* wop;
    const double* wopd;
    int32_t xwalls;        // 1: the mesh has isothermal or moving wall faces
};

template <typename T>
struct DevState {
    double* Wd;   // [5][nc] master cell averages (FP64)
    T* X;         // [nc][Stride<T>::xs] working state W^n, grad W^n (cell-major for neighbour gathers)
    T* Xs;        // [nc][Stride<T>::xs] stage state W*, grad W*
    double* S;    // [5][nc] saved stage-1 flux term
    T* G;         // [15][nc] saved stage-1 gradient term
    T* slopes;    // [nc][15]
    T* poly;      // [nc][Stride<T>::poly]
    T* rec;       // [nf][40]
    double* ctrl; // [CTRL_N] global controls (dt_fixed, t_end)
    double* case_t;   // [ncase] time of each case
    double* case_dt;  // [ncase] step of each case for the current step
    unsigned long long* case_dtmin;  // [ncase] bits of the minimum local dt (atomicMin)
    double* part; // [n_part_blocks][PART_N] residual sums per block
    int32_t* err;
};

struct HostPhys {
    double gamma, cfl, mu, eps_weno, tau_eps, tau_c;
    int weno, order, smooth, viscous;
    double prf;    // Pr fix factor 1/Pr - 1 (0: none)
    double twall;     // isothermal wall temperature
    double uwall[3];  // moving wall velocity
};

template <typename T>
struct Launch {
    // stage pieces
    // fin (may be NULL): block 0 first turns the per-block minima into the
    // step's dt (the time-step rule's global minimum, t_end clipping)
    struct Finalize {
        unsigned long long* dtmin;
        double* case_t;
        double* case_dt;
        int32_t ncase;
        double cfl;
        const double* ctrl;
    };
    static cudaError_t slopes(const DevMesh<T>& m, const T* X, T* slopes, const Finalize* fin,
                              cudaStream_t s);
    // slopes_in (may be NULL): the step-1 slopes of every cell from a slopes
    // pass; without it the kernel computes its own and its neighbours' slopes.
    // slopes_out (may be NULL) receives the cell's own step-1 slopes.
    // err: ERR_TIMEOUT is or-ed in if a block's bounded wait for its tile
    // gave up
    static cudaError_t recon(const DevMesh<T>& m, const HostPhys& p, const T* X, const T* slopes_in,
                             T* slopes_out, T* poly, int32_t* fallback, const Finalize* fin,
                             int32_t* err, cudaStream_t s);
    // case_dt: per-case step (NULL: dt_override for every face)
    // variant: 1 = 3 blocks per SM (FP32), 0 = 2 blocks per SM; ignored in FP64
    static cudaError_t flux(const DevMesh<T>& m, const HostPhys& p, const T* X, const T* poly, T* rec,
                            const double* case_dt, double dt_override, int stage, cudaStream_t s,
                            int variant = 1);
    static cudaError_t update1(const DevMesh<T>& m, const HostPhys& p, const DevState<T>& st, cudaStream_t s);
    static cudaError_t update2(const DevMesh<T>& m, const HostPhys& p, const DevState<T>& st,
                               cudaStream_t s);
    static cudaError_t dt_partials(const DevMesh<T>& m, const HostPhys& p, const T* X,
                                   double* part, cudaStream_t s);
    // per-case minima of the local limits of X into case_dtmin (reset first)
    static cudaError_t init_dtmin(const DevMesh<T>& m, const HostPhys& p, const T* X,
                                  unsigned long long* case_dtmin, cudaStream_t s);
    // X = [W | grad W] per cell from FP64 component-major W[5][nc], dW[15][nc]
    // (cperm, may be NULL: device cell -> cell of W, dW)
    static cudaError_t pack(const double* W, const double* dW, T* X, int64_t nc, cudaStream_t s,
                            const int32_t* cperm = nullptr);
    // FP64 component-major dW[15][nc] from X (in the order of cperm's cells)
    static cudaError_t unpack_grad(const T* X, double* dW, int64_t nc, cudaStream_t s,
                                   const int32_t* cperm = nullptr);
    // conversions for diagnostics
    static cudaError_t to_double(const T* in, double* out, int64_t n, cudaStream_t s);
    static cudaError_t from_double(const double* in, T* out, int64_t n, cudaStream_t s);
    // face records in device order -> FP64 in canonical order (perm: device -> canonical).
    // FP32 stage-1 records hold the interface states and fluxes relative to
    // the mean W_m of the two cells' averages (Stride comment above); with m
    // and X given, W_m sum_k w_k n and the flux terms (dt / 2) A F_n(W_m),
    // dt A F_n(W_m) are added back so that the output is the record of the
    // definition.
    static cudaError_t rec_to_double(const T* rec, const int32_t* perm, double* out, int64_t nf, int nr,
                                     const DevMesh<T>* m, const T* X, double gm1, double dt, cudaStream_t s);
    // padded reconstruction records -> compact FP64 [nc][50] in centroid-monomial form
    // (rows in the order of cperm's cells)
    static cudaError_t poly_to_double(const T* in, double* out, int64_t nc, cudaStream_t s,
                                      const int32_t* cperm = nullptr);
};

// Local time-step limit of one cell (Sec. 5, Eq. time-step, without C_CFL):
// dr / (|U| + a), and dr^2 / (3 nu) if viscous, from its averages Wv[5],
// in the working precision T.
#ifdef __CUDACC__
template <typename T>
__device__ __forceinline__ T local_dt(const T* Wv, T dr, const HostPhys& p) {
    const T ir = T(1) / Wv[0];
    const T u = Wv[1] * ir, v = Wv[2] * ir, w = Wv[3] * ir;
    const T q = u * u + v * v + w * w;
    const T pr = T(p.gamma - 1.0) * (Wv[4] - T(0.5) * Wv[0] * q);
    const T a = sqrt(T(p.gamma) * pr * ir);
    T d = dr / (sqrt(q) + a);
    if (p.viscous && p.mu > 0.0) {
        const T dv = dr * dr * Wv[0] / (T(3.0 * p.mu));
        d = d < dv ? d : dv;
    }
    return d;
}
#endif

// Device buffers of the adjoint sweep (FP64): the two stages' reconstruction
// records, the per-cell record adjoints (up to 40), the per-face adjoints of
// both cells' reconstruction coefficients [nf][2][50] (through the point
// input adjoints [nf][3][40]), their per-cell sums
// [nc][50], stencil adjoints [nc][5][16] and own parts [nc][5], the working
// state adjoints of the stage and of the step [nc][XS], the reverse face
// slots [4][nc] and the positivity-fallback flags of both stages [2][nc].
struct AdjBuffers {
    const double* poly1;
    const double* poly2;
    double *src, *lx, *lpf, *lp, *ld, *own, *lXs, *lX1;
    double *lbn, *lds;  // WENO only: neighbour-slope adjoints [nc][5][4][3], [nc][5][4]
    double* lwo;        // open-face ghost adjoints [nf][5]
    const int8_t* rev;
    int32_t* fallback;
};
// [ncomp][nc] FP64 arrays between device cell order and the caller's
// (cperm: device cell -> caller's cell; to_public 1: out[cperm[d]] = in[d])
cudaError_t launch_cells_perm(const double* in, double* out, int64_t nc, int ncomp, const int32_t* cperm,
                              int to_public, cudaStream_t s);
// out row r = in row map[r] for rows of width_words 4-byte words
cudaError_t launch_rows_gather(const void* in, void* out, int64_t nrows, int width_words, const int32_t* map,
                               cudaStream_t s);
// the one-launch stage's grid barrier on a barrier nothing completes: each
// of two blocks polls `limit` times, gives up and sets ERR_TIMEOUT
cudaError_t launch_grid_barrier_probe(unsigned* gbar, int32_t* err, int limit, cudaStream_t s);
// the averages W [5][nc] of an FP64 working state X [nc][XS]
cudaError_t launch_unpack_avg(const double* X, double* W, int64_t nc, cudaStream_t s);
// one stage of the FP32-bulk step (reconstruction with the neighbours'
// slopes recomputed, face flux, cell update) as one persistent launch with
// grid-wide barriers; gbar: 2 unsigned words of device scratch (reset by the
// launch); fin (stage 1, may be NULL) as for the reconstruction
cudaError_t launch_stage(const DevMesh<float>& m, const HostPhys& p, const DevState<float>& st, int stage,
                         const Launch<float>::Finalize* fin, unsigned* gbar, cudaStream_t s);
// a bounded mbarrier wait that gives up (nothing completes it): sets ERR_TIMEOUT
cudaError_t launch_wait_probe(int32_t* err, int tries, cudaStream_t s);

// lambda (W^n, grad W^n) from lambda (W^{n+1}, grad W^{n+1}) for one step
// with the frozen time step dt (public [component][cell] FP64 layouts)
cudaError_t adjoint_reverse(const DevMesh<double>& m, const HostPhys& p, double dt, const AdjBuffers& b,
                            const double* X1, const double* X2, const double* lW, const double* ldW, double* oW,
                            double* odW, cudaStream_t s);

// sets dt_fixed and t_end; with reset_time also zeroes the case times and
// steps and sets the case minima to +inf
cudaError_t launch_set_control(double* ctrl, double* case_t, double* case_dt,
                               unsigned long long* case_dtmin, int32_t ncase, double dt_fixed,
                               double t_end, int reset_time, cudaStream_t s);
int update_blocks(int64_t nc);

}  // namespace gks
