// gks_flux_xw.cu -- the FP32 face-flux instances for meshes with isothermal
// or moving wall faces (Sec. 4.4 ghosts of those walls compiled in), kept
// apart so that the common instances carry no code for them and the two
// sets compile in parallel.
#include <cuda_runtime.h>

#include "gks_flux.cuh"

namespace gks {

cudaError_t launch_flux_xw(const DevMesh<float>& m, const Phys<float>& ph, const float* W, const float* poly,
                           float* rec, const double* ctrl, double dt_override, int stage, cudaStream_t s,
                           int variant, bool prf) {
    const unsigned grid = (unsigned)((m.nf + FLUX_FACES - 1) / FLUX_FACES);
    auto go = [&](auto kernel) { kernel<<<grid, 2 * FP_GP, 0, s>>>(m, ph, W, poly, rec, ctrl, dt_override); };
    if (variant == 1) {
        if (stage == 1)
            prf ? go(k_flux<float, 40, 3, true, true>) : go(k_flux<float, 40, 3, false, true>);
        else
            prf ? go(k_flux<float, 20, 3, true, true>) : go(k_flux<float, 20, 3, false, true>);
    } else {
        if (stage == 1)
            prf ? go(k_flux<float, 40, 2, true, true>) : go(k_flux<float, 40, 2, false, true>);
        else
            prf ? go(k_flux<float, 20, 2, true, true>) : go(k_flux<float, 20, 2, false, true>);
    }
    return cudaGetLastError();
}

}  // namespace gks
