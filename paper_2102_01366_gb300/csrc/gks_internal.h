// gks_internal.h -- host-side objects shared by the translation units of
// libgks (mesh setup, stencil construction, device state).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/gks.h"

struct gks_mesh {
    int64_t nv = 0, nc = 0, nf = 0, nbf = 0;
    int32_t ncase = 1;
    std::vector<double> period;    // ncase*3, 0 on a non-periodic axis
    std::vector<int32_t> cell_case;  // nc (all 0 for one case)
    const double* per(int64_t c) const { return &period[(size_t)cell_case[c] * 3]; }
    std::vector<double> xyz;      // nv*3
    std::vector<int64_t> tet;     // nc*4
    std::vector<int8_t> shift;    // nc*12
    // connectivity
    std::vector<int64_t> face_v;     // nf*3 ascending vertex ids
    std::vector<int64_t> face_lr;    // nf*2
    std::vector<int64_t> nbr;        // nc*4
    std::vector<int32_t> nbr_img;    // nc*12 image shift, own frame -> neighbour
    std::vector<int64_t> csr_face;   // nc*4
    std::vector<int8_t> csr_sign;    // nc*4
    std::vector<int8_t> bkind;       // nf, GKS_BC_* of boundary faces (0 elsewhere)
    // FP64 geometry
    std::vector<double> vol, cen, mom2, dr;       // nc, nc*3, nc*6, nc
    std::vector<double> farea, fnorm, gp_l, gp_r; // nf, nf*3, nf*9, nf*9
    // stencils
    bool has_stencils = false;
    int64_t n_singular = 0;
    std::vector<double> M1, M2;   // nc*12, nc*144
    std::vector<uint8_t> singular;
};

namespace gks {
void set_error(const std::string& msg);
gks_status build_mesh(gks_mesh& m);      // topology + geometry
gks_status build_stencils(gks_mesh& m);  // M1, M2
bool cell_linear_fit(const gks_mesh& m, int64_t c, double* M2);  // boundary cells, linear weights
// Sec. 4.4 constrained operators of a cell with non-slip adiabatic wall
// faces (see gks_stencil.cpp); false when it has none or they cannot be built
bool cell_wall_stencil(const gks_mesh& m, int64_t c, double* W2, double* W1);
bool has_wall_face(const gks_mesh& m, int64_t c);
}  // namespace gks
