// lbm_core.cuh -- per-site arithmetic of the multirange Shan-Chen lattice Boltzmann step
// (Sbragaglia, Benzi, Bernaschi, Succi, arXiv:1402.6019), shared by every step kernel.
//
// Everything here is __host__ __device__ and free of CUDA intrinsics so the same arithmetic
// can be compiled for the host.  Kernels gather the neighbourhood values (by warp shuffles
// or from shared memory) and call these functions.
#pragma once

#include <math.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define LBM_HD __host__ __device__ __forceinline__
#else
#define LBM_HD inline
#endif

namespace lbm {

// ---------------------------------------------------------------------------------------
// Lattice.  D2Q9 velocities in the order c0 = (0,0), c1 = (1,0), c2 = (0,1), c3 = (-1,0),
// c4 = (0,-1), c5 = (1,1), c6 = (-1,1), c7 = (-1,-1), c8 = (1,-1): c1..c8 are also the
// first interaction belt, and Appendix A's pair terms (c13 = c5 - c3 = c1 - c7, ...) hold.
// ---------------------------------------------------------------------------------------
LBM_HD constexpr int cx(int l) { return l == 1 || l == 5 || l == 8 ? 1 : (l == 3 || l == 6 || l == 7 ? -1 : 0); }
LBM_HD constexpr int cz(int l) { return l == 2 || l == 5 || l == 6 ? 1 : (l == 4 || l == 7 || l == 8 ? -1 : 0); }
LBM_HD constexpr int opp(int l) { return l == 0 ? 0 : (l <= 4 ? (l + 1) % 4 + 1 : (l - 5 + 2) % 4 + 5); }
// rest weights of D2Q9: 4/9, 1/9 (axis), 1/36 (diagonal)
template <typename T> LBM_HD constexpr T wlb(int l) { return l == 0 ? T(4) / T(9) : (l <= 4 ? T(1) / T(9) : T(1) / T(36)); }

// Per-step constants, passed to kernels by value (they live in the kernel-parameter
// constant bank).  Force tables are indexed by the neighbour offset (dz + 2) * 5 + dx + 2.
template <typename T>
struct StepConst {
    int nx, nz, pitch, ns;
    int zbc;        // 0 periodic, 1 bounce-back walls
    int psi_form;   // 0 psi = 1 - exp(-rho/rho0), 1 psi = rho
    int psi_wall;   // 0 mirror, 1 zero
    int pad0;
    long long plane;          // elements of one population plane (nz * pitch)
    T omega[2], tau[2], rho_ref[2], inv_rho0[2], rho0[2];
    T g;                      // body acceleration along x
    T wall_u[2];              // bottom, top wall velocity (x)
    T kx[2][25], kz[2][25];   // K_s(|c|^2) c for the intra-species force
    T sq[2][9];               // App. A shell prefactors x K_s by |c|^2
    T kcx[9], kcz[9];         // G_AB w8(|c|^2) c for the cross force, (dz+1)*3 + dx+1
    T sc[3];                  // G_AB w8(|c|^2) / 2 for the cross stress, by |c|^2 = 1, 2
    T kin[2];                 // (tau_s - 1/2)^2 of the Sec. III stress
};

// Pseudopotential of Sec. IV, psi = 1 - exp(-rho/rho0) (or psi = rho).  FP32 on the device
// uses the hardware exponential (absolute error ~1e-7 in psi, inside the FP32 mode's budget).
LBM_HD float psi_of(const StepConst<float>& C, int s, float rho) {
#if defined(__CUDA_ARCH__)
    return C.psi_form == 1 ? rho : 1.0f - __expf(-rho * C.inv_rho0[s]);
#else
    return C.psi_form == 1 ? rho : -expm1f(-rho * C.inv_rho0[s]);
#endif
}
LBM_HD double psi_of(const StepConst<double>& C, int s, double rho) {
    return C.psi_form == 1 ? rho : 1.0 - exp(-rho / C.rho0[s]);
}

// ---------------------------------------------------------------------------------------
// Eq. FORCE: F = -psi(x) sum_{l=1..24} K(|c_l|^2) psi(x + c_l) c_l, with
// K = G1 w + G2 p folded into the tables kx/kz.  p[dz+2][dx+2] = psi(x+dx, z+dz).  Antipodal
// links have opposite c, so the sum runs over the 12 differences psi(c) - psi(-c), gathered
// shell by shell and scaled once per shell: kx at (1,0), (1,1), (2,0), (1,2), (2,2) holds K(1),
// K(2), 2 K(4), K(5), 2 K(8).
// ---------------------------------------------------------------------------------------
template <typename T>
LBM_HD void intra_force(const StepConst<T>& C, int s, const T (&p)[5][5], T& fx, T& fz) {
#define LBM_Q(dx, dz) p[(dz) + 2][(dx) + 2]
    const T d10 = LBM_Q(1, 0) - LBM_Q(-1, 0), d01 = LBM_Q(0, 1) - LBM_Q(0, -1);
    const T d11 = LBM_Q(1, 1) - LBM_Q(-1, -1), e11 = LBM_Q(-1, 1) - LBM_Q(1, -1);
    const T d20 = LBM_Q(2, 0) - LBM_Q(-2, 0), d02 = LBM_Q(0, 2) - LBM_Q(0, -2);
    const T d21 = LBM_Q(2, 1) - LBM_Q(-2, -1), e21 = LBM_Q(-2, 1) - LBM_Q(2, -1);
    const T d12 = LBM_Q(1, 2) - LBM_Q(-1, -2), e12 = LBM_Q(-1, 2) - LBM_Q(1, -2);
    const T d22 = LBM_Q(2, 2) - LBM_Q(-2, -2), e22 = LBM_Q(-2, 2) - LBM_Q(2, -2);
    const T* k = C.kx[s];
    const T k1 = k[13], k2 = k[18], k4 = k[14], k5 = k[23], k8 = k[24];
    // shell |c|^2 = 5: the links (2,1), (-2,1), (1,2), (-1,2)
    const T x5 = T(2) * (d21 - e21) + (d12 - e12);
    const T z5 = T(2) * (d12 + e12) + (d21 + e21);
    const T sx = ((k1 * d10 + k2 * (d11 - e11)) + (k4 * d20 + k5 * x5)) + k8 * (d22 - e22);
    const T sz = ((k1 * d01 + k2 * (d11 + e11)) + (k4 * d02 + k5 * z5)) + k8 * (d22 + e22);
    fx = -LBM_Q(0, 0) * sx;
    fz = -LBM_Q(0, 0) * sz;
#undef LBM_Q
}

// ---------------------------------------------------------------------------------------
// Appendix A: interaction stress of one species, shells |c|^2 = 1, 2 (node products),
// 4 and 8 (node and half-link products), 5 (node products and the c13..c16 pair terms).
// sq[q] already holds (1/2 or 1/4) * (G1 w(q) + G2 p(q)).  Adds into (sxx, szz, sxz).
// ---------------------------------------------------------------------------------------
template <typename T>
LBM_HD void intra_stress(const StepConst<T>& C, int s, const T (&p)[5][5], T& sxx, T& szz, T& sxz) {
#define LBM_P(dx, dz) p[(dz) + 2][(dx) + 2]
    const T p0 = LBM_P(0, 0);
    const T* q = C.sq[s];
    // |c|^2 = 1 and 2: node products
    const T d2 = LBM_P(1, 1) + LBM_P(-1, -1), a2 = LBM_P(-1, 1) + LBM_P(1, -1);
    const T n12x = q[1] * (LBM_P(1, 0) + LBM_P(-1, 0)) + q[2] * (d2 + a2);
    const T n12z = q[1] * (LBM_P(0, 1) + LBM_P(0, -1)) + q[2] * (d2 + a2);
    const T n12xz = q[2] * (d2 - a2);
    // |c|^2 = 4: node products and half-link products psi(x - c/2) psi(x + c/2)
    const T s4x = T(4) * q[4] * (p0 * (LBM_P(2, 0) + LBM_P(-2, 0)) + T(2) * LBM_P(-1, 0) * LBM_P(1, 0));
    const T s4z = T(4) * q[4] * (p0 * (LBM_P(0, 2) + LBM_P(0, -2)) + T(2) * LBM_P(0, -1) * LBM_P(0, 1));
    // |c|^2 = 5: node products over the 8 links (+-2,+-1), (+-1,+-2), and the pair terms of
    // links c13 = (2,1), c14 = (1,2), c15 = (-1,2), c16 = (-2,1)
    const T a21 = LBM_P(2, 1) + LBM_P(-2, -1), b21 = LBM_P(-2, 1) + LBM_P(2, -1);
    const T a12 = LBM_P(1, 2) + LBM_P(-1, -2), b12 = LBM_P(-1, 2) + LBM_P(1, -2);
    const T t13 = LBM_P(1, 1) * LBM_P(-1, 0) + LBM_P(1, 0) * LBM_P(-1, -1);
    const T t14 = LBM_P(1, 1) * LBM_P(0, -1) + LBM_P(0, 1) * LBM_P(-1, -1);
    const T t15 = LBM_P(0, 1) * LBM_P(1, -1) + LBM_P(-1, 1) * LBM_P(0, -1);
    const T t16 = LBM_P(-1, 1) * LBM_P(1, 0) + LBM_P(-1, 0) * LBM_P(1, -1);
    const T s5x = q[5] * (p0 * (T(4) * (a21 + b21) + (a12 + b12)) + (T(4) * (t13 + t16) + (t14 + t15)));
    const T s5z = q[5] * (p0 * ((a21 + b21) + T(4) * (a12 + b12)) + ((t13 + t16) + T(4) * (t14 + t15)));
    const T s5xz = q[5] * (T(2) * p0 * ((a21 - b21) + (a12 - b12)) + T(2) * ((t13 + t14) - (t15 + t16)));
    // |c|^2 = 8: node and half-link products over (+-2,+-2)
    const T a22 = LBM_P(2, 2) + LBM_P(-2, -2), b22 = LBM_P(-2, 2) + LBM_P(2, -2);
    const T ha = T(2) * LBM_P(-1, -1) * LBM_P(1, 1), hb = T(2) * LBM_P(-1, 1) * LBM_P(1, -1);
    const T s8 = T(4) * q[8] * (p0 * (a22 + b22) + (ha + hb));
    const T s8xz = T(4) * q[8] * (p0 * (a22 - b22) + (ha - hb));
    sxx += (p0 * n12x + s4x) + (s5x + s8);
    szz += (p0 * n12z + s4z) + (s5z + s8);
    sxz += (p0 * n12xz + s5xz) + s8xz;
#undef LBM_P
}

// ---------------------------------------------------------------------------------------
// Sec. IV cross repulsion (first belt, rho as the cross pseudopotential):
// F_A += -G_AB rho_A(x) sum_l w8 rho_B(x+c_l) c_l, and A <-> B.  r?[dz+1][dx+1].
// ---------------------------------------------------------------------------------------
template <typename T>
LBM_HD void cross_force(const StepConst<T>& C, const T (&ra)[3][3], const T (&rb)[3][3], T (&F)[2][2]) {
    // over the 4 antipodal differences of the first belt, shell by shell (kcx at (1,0), (1,1):
    // G_AB w8(1), G_AB w8(2))
    const T k1 = C.kcx[1 * 3 + 2], k2 = C.kcx[2 * 3 + 2];
    const T a10 = rb[1][2] - rb[1][0], a01 = rb[2][1] - rb[0][1];
    const T a11 = rb[2][2] - rb[0][0], b11 = rb[2][0] - rb[0][2];  // (1,1) and (-1,1)
    const T c10 = ra[1][2] - ra[1][0], c01 = ra[2][1] - ra[0][1];
    const T c11 = ra[2][2] - ra[0][0], e11 = ra[2][0] - ra[0][2];
    F[0][0] -= ra[1][1] * (k1 * a10 + k2 * (a11 - b11));
    F[0][1] -= ra[1][1] * (k1 * a01 + k2 * (a11 + b11));
    F[1][0] -= rb[1][1] * (k1 * c10 + k2 * (c11 - e11));
    F[1][1] -= rb[1][1] * (k1 * c01 + k2 * (c11 + e11));
}

// Cross-species stress, by analogy with App. A's first-belt shells: the pair product
// psi(x) psi(x+c) becomes rho_A(x) rho_B(x+c) + rho_B(x) rho_A(x+c).
template <typename T>
LBM_HD void cross_stress(const StepConst<T>& C, const T (&ra)[3][3], const T (&rb)[3][3], T& sxx, T& szz, T& sxz) {
    const T a0 = ra[1][1], b0 = rb[1][1];
#define LBM_PHI(dx, dz) (a0 * rb[(dz) + 1][(dx) + 1] + b0 * ra[(dz) + 1][(dx) + 1])
    const T s1x = LBM_PHI(1, 0) + LBM_PHI(-1, 0), s1z = LBM_PHI(0, 1) + LBM_PHI(0, -1);
    const T d = LBM_PHI(1, 1) + LBM_PHI(-1, -1), a = LBM_PHI(-1, 1) + LBM_PHI(1, -1);
#undef LBM_PHI
    sxx += C.sc[1] * s1x + C.sc[2] * (d + a);
    szz += C.sc[1] * s1z + C.sc[2] * (d + a);
    sxz += C.sc[2] * (d - a);
}

// ---------------------------------------------------------------------------------------
// Moments of Sec. II on stored values (deviations from W_l rho_ref, or plain values with
// rho_ref = 0): drho = sum f, j = sum f c.
// ---------------------------------------------------------------------------------------
template <typename T>
LBM_HD T sum9(const T (&f)[9]) {
    return ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
}
template <typename T>
LBM_HD void momentum9(const T (&f)[9], T& jx, T& jz) {
    jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    jz = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
}

// Equilibrium of Sec. II as a deviation from W_l rho_ref: W_l [drho + rho (3 cu + 9/2 cu^2 - 3/2 u^2)].
template <typename T>
LBM_HD T feq_dev(int l, T drho, T rho, T ux, T uz) {
    const T cu = T(cx(l)) * ux + T(cz(l)) * uz;
    const T usq = ux * ux + uz * uz;
    return wlb<T>(l) * (drho + rho * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * usq));
}

// Division and reciprocal: exact IEEE in FP64; in FP32 on the device the fast hardware
// approximation (a few ulp), well inside the FP32 mode's error budget.
LBM_HD double div_(double a, double b) { return a / b; }
LBM_HD float div_(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fdividef(a, b);
#else
    return a / b;
#endif
}

// The nine equilibria of Sec. II as deviations from W_l rho_ref, using the pair structure of
// D2Q9: l and its opposite share the even part W (drho + rho (9/2 cu^2 - 3/2 u^2)) and have
// odd parts +-3 W rho cu.
template <typename T>
LBM_HD void feq9_dev(T drho, T rho, T ux, T uz, T (&fe)[9]) {
    const T u15 = T(1.5) * (ux * ux + uz * uz);
    const T w1 = T(1) / T(9), w2 = T(1) / T(36);
    fe[0] = T(4) / T(9) * (drho - rho * u15);
    const T cu[4] = {ux, uz, ux + uz, uz - ux};  // pairs (1,3), (2,4), (5,7), (6,8)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const T w = k < 2 ? w1 : w2;
        const T even = w * (drho + rho * (T(4.5) * cu[k] * cu[k] - u15));
        const T odd = w * T(3) * rho * cu[k];
        const int lp = k < 2 ? k + 1 : k + 3;  // 1, 2, 5, 6
        fe[lp] = even + odd;
        fe[opp(lp)] = even - odd;
    }
}

// Shifted-velocity BGK collision of all species at one site (Eq. LB with u_eq = u' + tau F /
// rho, u' the common velocity sum_s j_s/tau_s / sum_s rho_s/tau_s).  f is overwritten with the
// post-collision values f + omega (feq - f) = (1 - omega) f + omega feq.  omega is folded into
// the equilibrium's coefficients, and the pair structure of D2Q9 is used: l and its opposite
// share the even part omega W (drho + rho (9/2 cu^2 - 3/2 u^2)) and have odd parts
// +-3 omega W rho cu.  rho[s] is the full density, drho[s] the stored sum, ir[s] = 1/rho[s],
// (jx, jz) the momenta of the stored values.
template <typename T, int NS>
LBM_HD void collide(const StepConst<T>& C, T (&f)[NS][9], const T (&drho)[NS], const T (&rho)[NS],
                    const T (&ir)[NS], const T (&jx)[NS], const T (&jz)[NS], const T (&F)[NS][2]) {
    T nx_ = T(0), nz_ = T(0), den = T(0);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        nx_ += C.omega[s] * jx[s];
        nz_ += C.omega[s] * jz[s];
        den += C.omega[s] * rho[s];
    }
    const T iden = div_(T(1), den);
    const T upx = nx_ * iden, upz = nz_ * iden;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const T om = C.omega[s], keep = T(1) - om;
        const T tir = C.tau[s] * ir[s];
        const T ux = upx + F[s][0] * tir;
        const T uz = upz + F[s][1] * tir;
        const T u15 = T(1.5) * (ux * ux + uz * uz);
        const T b = om * rho[s];
        const T base = om * drho[s] - b * u15;  // omega (drho - 3/2 rho u^2)
        // even part e + c cu^2 and odd part d cu, axis (W = 1/9) and diagonal (W = 1/36) pairs
        const T e1 = base * T(1.0 / 9.0), c1 = b * T(0.5), d1 = b * T(1.0 / 3.0);
        const T e2 = base * T(1.0 / 36.0), c2 = b * T(0.125), d2 = b * T(1.0 / 12.0);
        f[s][0] = f[s][0] * keep + base * T(4.0 / 9.0);
        const T cu[4] = {ux, uz, ux + uz, uz - ux};  // pairs (1,3), (2,4), (5,7), (6,8)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const T even = k < 2 ? e1 + (c1 * cu[k]) * cu[k] : e2 + (c2 * cu[k]) * cu[k];
            const T odd = (k < 2 ? d1 : d2) * cu[k];
            const int lp = k < 2 ? k + 1 : k + 3;  // 1, 2, 5, 6
            f[s][lp] = (f[s][lp] * keep + even) + odd;
            f[s][opp(lp)] = (f[s][opp(lp)] * keep + even) - odd;
        }
    }
}

// Ladd's moving-wall bounce-back value for a population g_l (l pointing into a wall that
// moves with velocity uw along x): g_l - 2 W_l rho (c_l . U_w) / c_s^2.
template <typename T>
LBM_HD T bounce(int l, T g, T rho, T uw) {
    return g - T(6) * wlb<T>(l) * rho * T(cx(l)) * uw;
}

// Per-site observables that need the populations (before collision): the barycentric
// velocity (sum_s j_s + F_s/2) / sum_s rho_s, and the kinetic xz momentum flux, the xz second
// moment averaged over the collision of Eq. LB:
//   sum_s (1/2) (Pi_s + Pi*_s),  Pi*_s = (1 - omega_s) Pi_s + omega_s rho_s ueq_x ueq_z,
// i.e. sum_s (1 - omega_s/2) Pi_s + (omega_s/2) rho_s ueq_x ueq_z, where Pi_s = sum_l f_l c_lx c_lz
// (only the diagonal links have c_lx c_lz != 0; the rest weights cancel, so FP32 deviations
// give the same) and ueq_s = u' + tau_s F_s / rho_s the velocity of the shifted equilibrium
// (u' = sum_s omega_s j_s / sum_s omega_s rho_s), whose second moment is rho_s ueq_x ueq_z.
template <typename T, int NS>
LBM_HD void site_kinetics(const StepConst<T>& C, const T (&f)[NS][9], const T (&rho)[NS], const T (&ir)[NS],
                          const T (&jx)[NS], const T (&jz)[NS], const T (&F)[NS][2], T& ux, T& uz, T& pixz,
                          T& rtot, T& mx, T& mz) {
    mx = T(0);
    mz = T(0);
    rtot = T(0);
    T nx_ = T(0), nz_ = T(0), den = T(0);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        mx += jx[s] + T(0.5) * F[s][0];
        mz += jz[s] + T(0.5) * F[s][1];
        rtot += rho[s];
        nx_ += C.omega[s] * jx[s];
        nz_ += C.omega[s] * jz[s];
        den += C.omega[s] * rho[s];
    }
    const T irt = div_(T(1), rtot);
    ux = mx * irt;
    uz = mz * irt;
    const T iden = div_(T(1), den);
    const T upx = nx_ * iden, upz = nz_ * iden;
    pixz = T(0);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const T pi = (f[s][5] + f[s][7]) - (f[s][6] + f[s][8]);
        const T tir = C.tau[s] * ir[s];
        const T ex = upx + F[s][0] * tir, ez = upz + F[s][1] * tir;
        const T hom = T(0.5) * C.omega[s];
        pixz += (T(1) - hom) * pi + hom * rho[s] * ex * ez;
    }
}

// Index helpers.
LBM_HD int wrap_index(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}
// Reflection of a row index about the walls at z = -1/2 and z = n - 1/2.
LBM_HD int mirror_index(int z, int n) {
    int m = z % (2 * n);
    if (m < 0) m += 2 * n;
    return m >= n ? 2 * n - 1 - m : m;
}

// Row whose density stands at row r: periodic wrap, or with walls the mirror image (or -1
// for the zero ghost reading).  Rows inside the lattice take the branch without division.
template <typename T>
LBM_HD int source_row(const StepConst<T>& C, int r) {
    if (r >= 0 && r < C.nz) return r;
    if (C.zbc == 0) return wrap_index(r, C.nz);
    return C.psi_wall == 1 ? -1 : mirror_index(r, C.nz);
}

// Observable partial sums: per row (summed over x) and per column (summed over z).
enum { QR_UX = 0, QR_RHOA, QR_RHOB, QR_SXZ, QR_MX, QR_MZ, QR_WALLB, QR_WALLT, NQR };
enum { QC_PS = 0, QC_PXX, NQC };

}  // namespace lbm
