// lbm_consts.h -- host-side construction of the per-step constant tables (StepConst) from
// lbm_params: the interaction weights of Eq. FORCE / Appendix B folded with the couplings.
#pragma once

#include <string.h>

#include "lbm.h"
#include "lbm_core.cuh"

namespace lbm {

// ---------------------------------------------------------------------------------------
// Interaction weights by shell |c|^2.  Eq. FORCE fixes the ranges and App. B the
// constraints; these are the exact solutions (attraction: 6th-order isotropic on
// |c|^2 <= 4; repulsion: 6th- and 8th-order isotropic on |c|^2 <= 8; first belt: 4th order).
// ---------------------------------------------------------------------------------------
inline double w_attr_paper(int q) {
    switch (q) {
        case 1: return 4.0 / 15.0;
        case 2: return 1.0 / 10.0;
        case 4: return 1.0 / 120.0;
        default: return 0.0;
    }
}
inline double w_rep(int q) {
    switch (q) {
        case 1: return 4.0 / 21.0;
        case 2: return 4.0 / 45.0;
        case 4: return 1.0 / 60.0;
        case 5: return 2.0 / 315.0;
        case 8: return 1.0 / 5040.0;
        default: return 0.0;
    }
}
inline double w_belt1(int q) {
    switch (q) {
        case 1: return 1.0 / 3.0;
        case 2: return 1.0 / 12.0;
        default: return 0.0;
    }
}

template <typename T>
inline void fill_step_const(StepConst<T>& C, const lbm_params& p, int nx, int nz, int pitch, long long plane,
                            int ns, int zbc, const double rho_ref[2]) {
    memset(&C, 0, sizeof C);
    C.nx = nx;
    C.nz = nz;
    C.pitch = pitch;
    C.ns = ns;
    C.zbc = zbc;
    C.psi_form = p.psi_form;
    C.psi_wall = p.psi_wall;
    C.plane = plane;
    C.g = (T)p.body_force;
    C.wall_u[0] = (T)p.wall_u[0];
    C.wall_u[1] = (T)p.wall_u[1];
    const double wn = p.weight_norm;
    for (int s = 0; s < 2; ++s) {
        const int ps = s < ns ? s : 0;
        C.tau[s] = (T)p.tau[ps];
        C.omega[s] = (T)(1.0 / p.tau[ps]);
        C.rho0[s] = (T)p.rho0[ps];
        C.inv_rho0[s] = (T)(1.0 / p.rho0[ps]);
        C.rho_ref[s] = (T)rho_ref[ps];
        C.kin[s] = (T)((p.tau[ps] - 0.5) * (p.tau[ps] - 0.5));
        double K[9];
        for (int q = 0; q < 9; ++q) {
            const double wa = p.weight_preset == LBM_WEIGHTS_CHEM09 ? w_belt1(q) : w_attr_paper(q);
            K[q] = wn * (p.G1[ps] * wa + p.G2[ps] * w_rep(q));
            C.sq[s][q] = (T)((q <= 2 ? 0.5 : 0.25) * K[q]);
        }
        for (int dz = -2; dz <= 2; ++dz)
            for (int dx = -2; dx <= 2; ++dx) {
                const int q = dx * dx + dz * dz;
                C.kx[s][(dz + 2) * 5 + dx + 2] = (T)(K[q] * dx);
                C.kz[s][(dz + 2) * 5 + dx + 2] = (T)(K[q] * dz);
            }
    }
    const double gab = ns == 2 ? p.G_AB * wn : 0.0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dx = -1; dx <= 1; ++dx) {
            const int q = dx * dx + dz * dz;
            C.kcx[(dz + 1) * 3 + dx + 1] = (T)(gab * w_belt1(q) * dx);
            C.kcz[(dz + 1) * 3 + dx + 1] = (T)(gab * w_belt1(q) * dz);
        }
    C.sc[1] = (T)(0.5 * gab * w_belt1(1));
    C.sc[2] = (T)(0.5 * gab * w_belt1(2));
}

}  // namespace lbm
