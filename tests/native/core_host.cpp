// Host build of the library's per-site arithmetic (lbm_core.cuh + lbm_consts.h), so the
// tests can compare it with the oracle site by site without a GPU.
#include "lbm_consts.h"

using namespace lbm;

extern "C" int core_site(const lbm_params* p, int ns, const double* psi25, const double* rho9, double* F,
                         double* sint, double* scross) {
    StepConst<double> C;
    const double rr[2] = {0.0, 0.0};
    fill_step_const<double>(C, *p, 8, 8, 32, 256, ns, 0, rr);
    double Fs[2][2] = {{0, 0}, {0, 0}};
    for (int s = 0; s < ns; ++s) {
        double q[5][5];
        for (int dz = 0; dz < 5; ++dz)
            for (int dx = 0; dx < 5; ++dx) q[dz][dx] = psi25[s * 25 + dz * 5 + dx];
        intra_force(C, s, q, Fs[s][0], Fs[s][1]);
        double xx = 0, zz = 0, xz = 0;
        intra_stress(C, s, q, xx, zz, xz);
        sint[3 * s] = xx;
        sint[3 * s + 1] = zz;
        sint[3 * s + 2] = xz;
    }
    scross[0] = scross[1] = scross[2] = 0.0;
    if (ns == 2) {
        double ra[3][3], rb[3][3];
        for (int dz = 0; dz < 3; ++dz)
            for (int dx = 0; dx < 3; ++dx) {
                ra[dz][dx] = rho9[dz * 3 + dx];
                rb[dz][dx] = rho9[9 + dz * 3 + dx];
            }
        cross_force(C, ra, rb, Fs);
        cross_stress(C, ra, rb, scross[0], scross[1], scross[2]);
    }
    for (int s = 0; s < ns; ++s) {
        F[2 * s] = Fs[s][0];
        F[2 * s + 1] = Fs[s][1];
    }
    return 0;
}

// psi of one density with the library's formula
extern "C" double core_psi(const lbm_params* p, int s, double rho) {
    StepConst<double> C;
    const double rr[2] = {0.0, 0.0};
    fill_step_const<double>(C, *p, 8, 8, 32, 256, 2, 0, rr);
    return psi_of(C, s, rho);
}
