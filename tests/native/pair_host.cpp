// Host build of the two-species FP32 per-site arithmetic (lbm_pair.cuh), so the tests can compare
// it with the oracle site by site without a GPU.  The packed FP32 instructions it is written with
// get plain C++ stand-ins that round alike: per-lane add, multiply and fused multiply-add.
#include <cmath>

struct float2 {
    float x, y;
};
static inline float2 make_float2(float a, float b) { return float2{a, b}; }
static inline float2 __fadd2_rn(float2 a, float2 b) { return float2{a.x + b.x, a.y + b.y}; }
static inline float2 __fmul2_rn(float2 a, float2 b) { return float2{a.x * b.x, a.y * b.y}; }
static inline float2 __ffma2_rn(float2 a, float2 b, float2 c) {
    return float2{std::fma(a.x, b.x, c.x), std::fma(a.y, b.y, c.y)};
}
static inline float __fdividef(float a, float b) { return a / b; }
#define __device__
#define __forceinline__ inline

#include "lbm_consts.h"
#include "lbm_pair.cuh"

using namespace lbm;

// One site of a two-species lattice: psi25 = psi of both species on the 5 x 5 window
// ([s][dz + 2][dx + 2]), rho9 = rho of both species on the 3 x 3 window.  Outputs (FP64 copies of
// the FP32 results): F = intra + cross force from intra_force2, F2 = the same with force_stress2,
// sint = the App. A stresses of each species (sxx, szz, sxz) from force_stress2, scross = the
// cross stress (cross_stress2), psi = psi2 of the centre densities.
extern "C" int pair_site(const lbm_params* p, const double* psi25, const double* rho9, double* F, double* F2,
                         double* sint, double* scross, double* psi) {
    StepConst<float> C;
    const double rr[2] = {0.0, 0.0};
    fill_step_const<float>(C, *p, 8, 8, 32, 256, 2, 0, rr);
    PairConst K;
    fill_pair_const(K, C);
    f2 q[5][5], w[25];
    for (int dz = 0; dz < 5; ++dz)
        for (int dx = 0; dx < 5; ++dx) {
            q[dz][dx] = make_float2((float)psi25[dz * 5 + dx], (float)psi25[25 + dz * 5 + dx]);
            w[dz * 5 + dx] = q[dz][dx];
        }
    f2 r[3][3];
    for (int dz = 0; dz < 3; ++dz)
        for (int dx = 0; dx < 3; ++dx) r[dz][dx] = make_float2((float)rho9[dz * 3 + dx], (float)rho9[9 + dz * 3 + dx]);
    f2 fx, fz;
    intra_force2(K, q, fx, fz);
    cross_force2(K, r, fx, fz);
    f2 gx, gz, a, b, c;
    force_stress2<5>(K, w, gx, gz, a, b, c);
    cross_force2(K, r, gx, gz);
    const f2 out[2][2] = {{fx, fz}, {gx, gz}};
    for (int k = 0; k < 2; ++k) {
        double* d = k == 0 ? F : F2;
        d[0] = out[k][0].x;
        d[1] = out[k][1].x;
        d[2] = out[k][0].y;
        d[3] = out[k][1].y;
    }
    const f2 st[3] = {a, b, c};
    for (int i = 0; i < 3; ++i) {
        sint[i] = st[i].x;
        sint[3 + i] = st[i].y;
    }
    float sxx = 0.f, szz = 0.f, sxz = 0.f;
    cross_stress2(C, r, sxx, szz, sxz);
    scross[0] = sxx;
    scross[1] = szz;
    scross[2] = sxz;
    const f2 ps = psi2(C, K, r[1][1]);
    psi[0] = ps.x;
    psi[1] = ps.y;
    return 0;
}

// The shifted-velocity BGK collision of both species (collide2) at one site, as the step kernel
// runs it: populations stored as FP32 deviations from W_l rho_ref, momentum and density formed
// from them.  f18 = the populations of species A then B (FP64, before collision), F4 = the force
// (Fx, Fz of A, then of B); out18 receives the post-collision populations (deviation + W_l rho_ref).
extern "C" int pair_collide(const lbm_params* p, const double* rho_ref, const double* f18, const double* F4,
                            double* out18) {
    StepConst<float> C;
    fill_step_const<float>(C, *p, 8, 8, 32, 256, 2, 0, rho_ref);
    PairConst K;
    fill_pair_const(K, C);
    f2 fp[9];
    for (int l = 0; l < 9; ++l)
        fp[l] = make_float2((float)(f18[l] - wlb<double>(l) * rho_ref[0]), (float)(f18[9 + l] - wlb<double>(l) * rho_ref[1]));
    const f2 dr = sum9_2(fp);
    const f2 rh = add2(K.rho_ref, dr);
    const f2 ir = p2(__fdividef(1.f, rh.x), __fdividef(1.f, rh.y));
    f2 jx, jz;
    momentum9_2(fp, jx, jz);
    collide2(K, fp, dr, rh, ir, jx, jz, p2((float)F4[0], (float)F4[2]), p2((float)F4[1], (float)F4[3]));
    for (int l = 0; l < 9; ++l) {
        out18[l] = (double)fp[l].x + wlb<double>(l) * (double)C.rho_ref[0];
        out18[9 + l] = (double)fp[l].y + wlb<double>(l) * (double)C.rho_ref[1];
    }
    return 0;
}
