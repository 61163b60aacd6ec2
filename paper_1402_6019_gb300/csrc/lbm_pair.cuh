// lbm_pair.cuh -- the per-site arithmetic of the two-species FP32 step with the species in
// lockstep: a float2 holds (species A, species B), and Blackwell's packed FP32 instructions
// (__ffma2_rn, __fadd2_rn, __fmul2_rn) do both species' work in one instruction.  Same formulas
// as lbm_core.cuh (Eq. FORCE, the cross repulsion of Sec. IV, Appendix A's stresses, the shifted
// equilibrium and BGK relaxation of Sec. II); only the grouping of the arithmetic differs.
// Device-only.
#pragma once

#include "lbm_core.cuh"

namespace lbm {

using f2 = float2;

__device__ __forceinline__ f2 p2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ f2 sp(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 swap2(f2 a) { return make_float2(a.y, a.x); }

// Constant tables of the step as (A, B) pairs, built on the host from StepConst<float>.
struct PairConst {
    f2 kf[5];           // Eq. FORCE by shell: K_s(1), K_s(2), 2 K_s(4), K_s(5), 2 K_s(8)
    f2 kf5x2, kf5x2n, kf5n, kf8n;  // 2 K_s(5), -2 K_s(5), -K_s(5), -2 K_s(8)
    f2 kc[2];           // cross force by shell, both halves alike: G_AB w8(1), G_AB w8(2)
    f2 sq[9];           // App. A shell prefactors by |c|^2
    f2 omega, tau, rho_ref, nexp;  // nexp = -log2(e) / rho0 (psi = 1 - 2^(nexp rho))
    f2 kin;             // (tau - 1/2)^2
    f2 keep;            // 1 - omega
    f2 half_om;         // 1 - omega / 2
    f2 hom;             // omega / 2
};

// The pairs from the per-species tables (host).
inline void fill_pair_const(PairConst& K, const StepConst<float>& C) {
    // K_s(q) c_x of the links (1,0), (1,1), (2,0), (1,2), (2,2): exactly K_s(q) or 2 K_s(q)
    const int at[5] = {2 * 5 + 3, 3 * 5 + 3, 2 * 5 + 4, 4 * 5 + 3, 4 * 5 + 4};
    for (int k = 0; k < 5; ++k) K.kf[k] = make_float2(C.kx[0][at[k]], C.kx[1][at[k]]);
    K.kf5x2 = make_float2(2.0f * K.kf[3].x, 2.0f * K.kf[3].y);
    K.kf5x2n = make_float2(-K.kf5x2.x, -K.kf5x2.y);
    K.kf5n = make_float2(-K.kf[3].x, -K.kf[3].y);
    K.kf8n = make_float2(-K.kf[4].x, -K.kf[4].y);
    // G_AB w8(q) c_x of the links (1,0), (1,1)
    K.kc[0] = make_float2(C.kcx[1 * 3 + 2], C.kcx[1 * 3 + 2]);
    K.kc[1] = make_float2(C.kcx[2 * 3 + 2], C.kcx[2 * 3 + 2]);
    for (int q = 0; q < 9; ++q) K.sq[q] = make_float2(C.sq[0][q], C.sq[1][q]);
    K.omega = make_float2(C.omega[0], C.omega[1]);
    K.tau = make_float2(C.tau[0], C.tau[1]);
    K.rho_ref = make_float2(C.rho_ref[0], C.rho_ref[1]);
    const float log2e = 1.4426950408889634f;
    K.nexp = make_float2(-log2e * C.inv_rho0[0], -log2e * C.inv_rho0[1]);
    K.kin = make_float2(C.kin[0], C.kin[1]);
    K.keep = make_float2(1.0f - C.omega[0], 1.0f - C.omega[1]);
    K.half_om = make_float2(1.0f - 0.5f * C.omega[0], 1.0f - 0.5f * C.omega[1]);
    K.hom = make_float2(0.5f * C.omega[0], 0.5f * C.omega[1]);
}

// 2^a by the hardware approximation with subnormal results flushed to zero
__device__ __forceinline__ float ex2_ftz(float a) {
#ifdef __CUDA_ARCH__
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
#else
    return exp2f(a);
#endif
}

// Pseudopotential of Sec. IV for both species: psi = 1 - exp(-rho / rho0) (hardware exp2), or
// psi = rho.
__device__ __forceinline__ f2 psi2(const StepConst<float>& C, const PairConst& K, f2 rho) {
    if (C.psi_form == 1) return rho;
    const f2 a = mul2(rho, K.nexp);
    return p2(1.0f - ex2_ftz(a.x), 1.0f - ex2_ftz(a.y));
}

// Eq. FORCE for both species: F = -psi(x) sum_l K(|c_l|^2) psi(x + c_l) c_l.  The 24 links come
// in antipodal pairs with opposite c, so the sum runs over the differences psi(c) - psi(-c) of
// one link of each pair, gathered shell by shell (one coefficient per shell).
__device__ __forceinline__ void intra_force2(const PairConst& K, const f2 (&p)[5][5], f2& fx, f2& fz) {
#define LBM_Q(dx, dz) p[(dz) + 2][(dx) + 2]
    const f2 d10 = sub2(LBM_Q(1, 0), LBM_Q(-1, 0)), d01 = sub2(LBM_Q(0, 1), LBM_Q(0, -1));
    const f2 d11 = sub2(LBM_Q(1, 1), LBM_Q(-1, -1)), e11 = sub2(LBM_Q(-1, 1), LBM_Q(1, -1));
    const f2 d20 = sub2(LBM_Q(2, 0), LBM_Q(-2, 0)), d02 = sub2(LBM_Q(0, 2), LBM_Q(0, -2));
    const f2 d21 = sub2(LBM_Q(2, 1), LBM_Q(-2, -1)), e21 = sub2(LBM_Q(-2, 1), LBM_Q(2, -1));
    const f2 d12 = sub2(LBM_Q(1, 2), LBM_Q(-1, -2)), e12 = sub2(LBM_Q(-1, 2), LBM_Q(1, -2));
    const f2 d22 = sub2(LBM_Q(2, 2), LBM_Q(-2, -2)), e22 = sub2(LBM_Q(-2, 2), LBM_Q(2, -2));
    // shell |c|^2 = 5: the links (2,1), (1,2), (-1,2), (-2,1)
    const f2 x5 = fma2(sp(2.f), sub2(d21, e21), sub2(d12, e12));
    const f2 z5 = fma2(sp(2.f), add2(d12, e12), add2(d21, e21));
    f2 sx = mul2(K.kf[0], d10), sz = mul2(K.kf[0], d01);
    sx = fma2(K.kf[1], sub2(d11, e11), sx);
    sz = fma2(K.kf[1], add2(d11, e11), sz);
    sx = fma2(K.kf[2], d20, sx);
    sz = fma2(K.kf[2], d02, sz);
    sx = fma2(K.kf[3], x5, sx);
    sz = fma2(K.kf[3], z5, sz);
    sx = fma2(K.kf[4], sub2(d22, e22), sx);
    sz = fma2(K.kf[4], add2(d22, e22), sz);
    const f2 m = p2(-LBM_Q(0, 0).x, -LBM_Q(0, 0).y);
    fx = mul2(m, sx);
    fz = mul2(m, sz);
#undef LBM_Q
}

// Eq. FORCE and the Appendix A stresses of both species in one pass over the 5 x 5 psi window
// w (w[(dz + 2) * W + dx + 2] = psi(x + dx, z + dz), shared memory), for the observing passes:
// the sums of intra_force2 and of Appendix A's shell stresses (as lbm_core.cuh forms them per
// species).  The 16 values of the shells |c|^2 = 4, 5, 8 enter both only through the difference
// (force) and the sum (stress) of antipodal links, so they are read pair by pair and folded into
// the accumulators at once; only the inner 3 x 3 values, which the stresses' products need, are
// held throughout.  Returns the stresses as (A, B) pairs.
template <int W>
__device__ __forceinline__ void force_stress2(const PairConst& K, const f2* __restrict__ w, f2& fx, f2& fz,
                                              f2& sxx, f2& szz, f2& sxz) {
#define LBM_W(dx, dz) w[((dz) + 2) * W + (dx) + 2]
    const f2 p0 = LBM_W(0, 0);
    const f2 q10 = LBM_W(1, 0), qm10 = LBM_W(-1, 0), q01 = LBM_W(0, 1), q0m1 = LBM_W(0, -1);
    const f2 q11 = LBM_W(1, 1), qm1m1 = LBM_W(-1, -1), qm11 = LBM_W(-1, 1), q1m1 = LBM_W(1, -1);
    // force, shells 1 and 2
    const f2 d11 = sub2(q11, qm1m1), e11 = sub2(qm11, q1m1);
    f2 sx = fma2(K.kf[1], sub2(d11, e11), mul2(K.kf[0], sub2(q10, qm10)));
    f2 sz = fma2(K.kf[1], add2(d11, e11), mul2(K.kf[0], sub2(q01, q0m1)));
    // shells 4, 5, 8 pair by pair: force += K c (psi(c) - psi(-c)); stress accumulators of the
    // sums psi(c) + psi(-c): a4 (shell 4), a5x = 4 s21 + s12, a5z = s21 + 4 s12,
    // a5xz = a21 - b21 + a12 - b12, a8 = a22 + b22, a8xz = a22 - b22
    f2 a4x, a4z, a5x, a5z, a5xz, a8, a8xz;
    {
        const f2 u = LBM_W(2, 0), v = LBM_W(-2, 0);
        sx = fma2(K.kf[2], sub2(u, v), sx);
        a4x = add2(u, v);
    }
    {
        const f2 u = LBM_W(0, 2), v = LBM_W(0, -2);
        sz = fma2(K.kf[2], sub2(u, v), sz);
        a4z = add2(u, v);
    }
    {  // (2,1)
        const f2 u = LBM_W(2, 1), v = LBM_W(-2, -1), d = sub2(u, v), t = add2(u, v);
        sx = fma2(K.kf5x2, d, sx);
        sz = fma2(K.kf[3], d, sz);
        a5x = mul2(sp(4.f), t);
        a5z = t;
        a5xz = t;
    }
    {  // (-2,1)
        const f2 u = LBM_W(-2, 1), v = LBM_W(2, -1), d = sub2(u, v), t = add2(u, v);
        sx = fma2(K.kf5x2n, d, sx);
        sz = fma2(K.kf[3], d, sz);
        a5x = fma2(sp(4.f), t, a5x);
        a5z = add2(a5z, t);
        a5xz = sub2(a5xz, t);
    }
    {  // (1,2)
        const f2 u = LBM_W(1, 2), v = LBM_W(-1, -2), d = sub2(u, v), t = add2(u, v);
        sx = fma2(K.kf[3], d, sx);
        sz = fma2(K.kf5x2, d, sz);
        a5x = add2(a5x, t);
        a5z = fma2(sp(4.f), t, a5z);
        a5xz = add2(a5xz, t);
    }
    {  // (-1,2)
        const f2 u = LBM_W(-1, 2), v = LBM_W(1, -2), d = sub2(u, v), t = add2(u, v);
        sx = fma2(K.kf5n, d, sx);
        sz = fma2(K.kf5x2, d, sz);
        a5x = add2(a5x, t);
        a5z = fma2(sp(4.f), t, a5z);
        a5xz = sub2(a5xz, t);
    }
    {  // (2,2)
        const f2 u = LBM_W(2, 2), v = LBM_W(-2, -2), d = sub2(u, v), t = add2(u, v);
        sx = fma2(K.kf[4], d, sx);
        sz = fma2(K.kf[4], d, sz);
        a8 = t;
        a8xz = t;
    }
    {  // (-2,2)
        const f2 u = LBM_W(-2, 2), v = LBM_W(2, -2), d = sub2(u, v), t = add2(u, v);
        sx = fma2(K.kf8n, d, sx);
        sz = fma2(K.kf[4], d, sz);
        a8 = add2(a8, t);
        a8xz = sub2(a8xz, t);
    }
    const f2 m = p2(-p0.x, -p0.y);
    fx = mul2(m, sx);
    fz = mul2(m, sz);
    // stresses: shells 1 and 2, then the products of the inner values
    const f2 four = sp(4.f), two = sp(2.f);
    const f2 d2 = add2(q11, qm1m1), a2 = add2(qm11, q1m1), da = add2(d2, a2);
    const f2 n12x = fma2(K.sq[1], add2(q10, qm10), mul2(K.sq[2], da));
    const f2 n12z = fma2(K.sq[1], add2(q01, q0m1), mul2(K.sq[2], da));
    const f2 n12xz = mul2(K.sq[2], sub2(d2, a2));
    const f2 q4 = mul2(four, K.sq[4]);
    const f2 s4x = mul2(q4, fma2(p0, a4x, mul2(two, mul2(qm10, q10))));
    const f2 s4z = mul2(q4, fma2(p0, a4z, mul2(two, mul2(q0m1, q01))));
    const f2 t13 = fma2(q11, qm10, mul2(q10, qm1m1));
    const f2 t14 = fma2(q11, q0m1, mul2(q01, qm1m1));
    const f2 t15 = fma2(q01, q1m1, mul2(qm11, q0m1));
    const f2 t16 = fma2(qm11, q10, mul2(qm10, q1m1));
    const f2 t1316 = add2(t13, t16), t1415 = add2(t14, t15);
    const f2 s5x = mul2(K.sq[5], fma2(p0, a5x, fma2(four, t1316, t1415)));
    const f2 s5z = mul2(K.sq[5], fma2(p0, a5z, fma2(four, t1415, t1316)));
    const f2 s5xz = mul2(K.sq[5], mul2(two, fma2(p0, a5xz, sub2(add2(t13, t14), add2(t15, t16)))));
    const f2 ha = mul2(two, mul2(qm1m1, q11)), hb = mul2(two, mul2(qm11, q1m1));
    const f2 q8 = mul2(four, K.sq[8]);
    const f2 s8 = mul2(q8, fma2(p0, a8, add2(ha, hb)));
    const f2 s8xz = mul2(q8, fma2(p0, a8xz, sub2(ha, hb)));
    sxx = add2(fma2(p0, n12x, s4x), add2(s5x, s8));
    szz = add2(fma2(p0, n12z, s4z), add2(s5z, s8));
    sxz = add2(fma2(p0, n12xz, s5xz), s8xz);
#undef LBM_W
}

// Sec. IV cross repulsion for both species (first belt, rho as the cross pseudopotential):
// F_A += -G_AB rho_A(x) sum_l w8 rho_B(x + c_l) c_l, and A <-> B.  r[dz+1][dx+1] = (rho_A, rho_B).
// As in intra_force2, over the differences of antipodal links, shell by shell.
__device__ __forceinline__ void cross_force2(const PairConst& K, const f2 (&r)[3][3], f2& fx, f2& fz) {
    const f2 d10 = sub2(r[1][2], r[1][0]), d01 = sub2(r[2][1], r[0][1]);
    const f2 d11 = sub2(r[2][2], r[0][0]), e11 = sub2(r[2][0], r[0][2]);  // (1,1), (-1,1)
    const f2 sx = fma2(K.kc[1], sub2(d11, e11), mul2(K.kc[0], d10));
    const f2 sz = fma2(K.kc[1], add2(d11, e11), mul2(K.kc[0], d01));
    // species A takes the sums over rho_B, species B those over rho_A
    const f2 m = p2(-r[1][1].x, -r[1][1].y);
    fx = fma2(m, swap2(sx), fx);
    fz = fma2(m, swap2(sz), fz);
}

// Cross-species stress (the pair product psi(x) psi(x + c) read as rho_A(x) rho_B(x + c) +
// rho_B(x) rho_A(x + c)); returns the sums into scalars.
__device__ __forceinline__ void cross_stress2(const StepConst<float>& C, const f2 (&r)[3][3], float& sxx, float& szz,
                                              float& sxz) {
    const f2 ba = swap2(r[1][1]);  // (rho_B(x), rho_A(x)): phi(c) = ba . r(c)
    const f2 e1x = mul2(ba, add2(r[1][2], r[1][0]));
    const f2 e1z = mul2(ba, add2(r[2][1], r[0][1]));
    const f2 ed = mul2(ba, add2(r[2][2], r[0][0]));
    const f2 ea = mul2(ba, add2(r[2][0], r[0][2]));
    const float s1x = e1x.x + e1x.y, s1z = e1z.x + e1z.y, d = ed.x + ed.y, a = ea.x + ea.y;
    sxx += C.sc[1] * s1x + C.sc[2] * (d + a);
    szz += C.sc[1] * s1z + C.sc[2] * (d + a);
    sxz += C.sc[2] * (d - a);
}

// In sum9's order (lbm_core.cuh): a site's density is the same number whether the tile that holds
// it forms it (here) or a neighbouring tile forms it for its halo (per species, sum9).
__device__ __forceinline__ f2 sum9_2(const f2 (&f)[9]) {
    return add2(add2(add2(add2(f[0], f[1]), add2(f[2], f[3])), add2(add2(f[4], f[5]), add2(f[6], f[7]))), f[8]);
}
__device__ __forceinline__ void momentum9_2(const f2 (&f)[9], f2& jx, f2& jz) {
    jx = add2(add2(sub2(f[1], f[3]), sub2(f[5], f[6])), sub2(f[8], f[7]));
    jz = add2(add2(sub2(f[2], f[4]), sub2(f[5], f[7])), sub2(f[6], f[8]));
}

// Shifted-velocity BGK collision of both species (Eq. LB, Sec. II), f overwritten with
// (1 - omega) f + omega feq; omega folded into the equilibrium's coefficients and the pair
// structure of D2Q9 used as in lbm_core.cuh's collide.
__device__ __forceinline__ void collide2(const PairConst& K, f2 (&f)[9], f2 drho, f2 rho, f2 ir, f2 jx, f2 jz, f2 Fx,
                                         f2 Fz) {
    const f2 wj = mul2(K.omega, jx), wk = mul2(K.omega, jz), wr = mul2(K.omega, rho);
    const float iden = __fdividef(1.0f, wr.x + wr.y);
    const f2 up = sp((wj.x + wj.y) * iden), vp = sp((wk.x + wk.y) * iden);
    const f2 tir = mul2(K.tau, ir);
    const f2 ux = fma2(Fx, tir, up);
    const f2 uz = fma2(Fz, tir, vp);
    const f2 u15 = mul2(sp(1.5f), fma2(ux, ux, mul2(uz, uz)));
    const f2 b = mul2(K.omega, rho);
    const f2 base = sub2(mul2(K.omega, drho), mul2(b, u15));  // omega (drho - 3/2 rho u^2)
    const f2 e1 = mul2(base, sp(1.0f / 9.0f)), c1 = mul2(b, sp(0.5f)), d1 = mul2(b, sp(1.0f / 3.0f));
    const f2 e2 = mul2(base, sp(1.0f / 36.0f)), c2 = mul2(b, sp(0.125f)), d2 = mul2(b, sp(1.0f / 12.0f));
    f[0] = fma2(f[0], K.keep, mul2(base, sp(4.0f / 9.0f)));
    const f2 cu[4] = {ux, uz, add2(ux, uz), sub2(uz, ux)};  // pairs (1,3), (2,4), (5,7), (6,8)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const f2 even = k < 2 ? fma2(mul2(c1, cu[k]), cu[k], e1) : fma2(mul2(c2, cu[k]), cu[k], e2);
        const f2 odd = mul2(k < 2 ? d1 : d2, cu[k]);
        const int lp = k < 2 ? k + 1 : k + 3;
        f[lp] = add2(fma2(f[lp], K.keep, even), odd);
        f[opp(lp)] = sub2(fma2(f[opp(lp)], K.keep, even), odd);
    }
}

}  // namespace lbm
