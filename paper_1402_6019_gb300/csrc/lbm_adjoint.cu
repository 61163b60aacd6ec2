// lbm_adjoint.cu -- discrete adjoint of the time step (periodic lattice), in FP64 or FP32.
//
// The step maps the post-streaming populations f_n to f_{n+1} = S(f_n; theta):
//   rho_s = sum_l f_l, j_s = sum_l f_l c_l (Sec. II); psi_s = psi(rho_s) (Sec. IV);
//   F_s = -psi_s(x) sum_c (G1_s w(c) + G2_s p(c)) psi_s(x + c) c            (Eq. FORCE)
//         - G_AB rho_s(x) sum_c w8(c) rho_s'(x + c) c + rho_s g x            (Sec. IV);
//   u' = sum_s j_s / tau_s / sum_s rho_s / tau_s, u_s = u' + tau_s F_s / rho_s;
//   feq_l = W_l rho_s (1 + 3 c.u_s + 9/2 (c.u_s)^2 - 3/2 u_s.u_s);
//   g_l = f_l - (f_l - feq_l) / tau_s (Eq. LB);  f_{n+1}(x + c_l, l) = g_l(x).
// Given lam_{n+1} = dJ/df_{n+1}, three kernels form lam_n = dJ/df_n and the derivatives with
// respect to theta = (G1 A, G1 B, G2 A, G2 B, G_AB, tau A, tau B, g) by applying the transposed
// derivative of each stage in reverse order:
//   k_adj_moments  rho, j and psi of the state f_n (the linearisation point) -- for the first
//                  step of a sweep; for the others k_adj_final of the step before forms them;
//   k_adj_local    the force at the site (from its neighbours' psi and rho), then streaming
//                  transposed (a gather of lam_{n+1}), relaxation, equilibrium, shifted and
//                  common velocity transposed: dJ/dF_s, the site's own share of dJ/drho_s and
//                  dJ/dj_s, and every parameter derivative of the site;
//   k_adj_final    the neighbour shares of the force transposed (each site gathers what the
//                  forces at x - c owe to its psi and rho), the pseudopotential and the
//                  moments: lam_n; and the moments of f_{n-1} for the next step back.
// T is the precision of the states and of lam (FP64, or FP32 for FP32 forward runs).  The
// parameter derivatives are summed per block (FP64, or double-float pairs in FP32 mode), kept
// per block across the steps of a call, then summed over the blocks in FP64 in a fixed order.
#include "lbm_consts.h"
#include "lbm_internal.h"
#include "lbm_reduce.cuh"

namespace lbm {

namespace {

constexpr int AT = 256;  // threads per block of the objective and sum kernels
constexpr int ST = 128;  // threads per block of the per-step kernels (more blocks on small lattices)
constexpr int NPAR = 8;

// (dx, dz) of the 24 interaction links, first belt first (|c|^2 = 1, 2), then 4, 5, 8; constant
// expressions, so an unrolled loop over the links folds them
LBM_HD constexpr int LKX(int k) {
    constexpr int t[24] = {1, 0, -1, 0, 1, -1, -1, 1, 2, 0, -2, 0, 2, 1, -1, -2, -2, -1, 1, 2, 2, -2, -2, 2};
    return t[k];
}
LBM_HD constexpr int LKZ(int k) {
    constexpr int t[24] = {0, 1, 0, -1, 1, 1, -1, -1, 0, 2, 0, -2, 1, 2, 2, 1, -1, -2, -2, -1, 2, 2, -2, -2};
    return t[k];
}

// Periodic coordinate v = c + d, |d| <= 2, of a lattice of n sites along that axis.
__device__ __forceinline__ int wrap2(int v, int n) {
    if (n < 3) return ((v % n) + n) % n;  // uniform branch: only tiny lattices wrap more than once
    return v < 0 ? v + n : (v >= n ? v - n : v);
}

// Site indices of the 5 x 5 neighbourhood of (x, z): xo[dx + 2] + zo[dz + 2].
struct Nbr {
    int xo[5], zo[5];
    __device__ __forceinline__ Nbr(int x, int z, int nx, int nz) {
#pragma unroll
        for (int d = 0; d < 5; ++d) {
            xo[d] = wrap2(x + d - 2, nx);
            zo[d] = wrap2(z + d - 2, nz) * nx;
        }
    }
    __device__ __forceinline__ long long at(int dx, int dz) const { return (long long)zo[dz + 2] + xo[dx + 2]; }
};

template <typename T>
struct AdjC {
    int nx, nz, ns, psi_form;
    T wa[9], wr[9], wc[9];  // by |c|^2, weight_norm included
    T G1[2], G2[2], tau[2], itau[2], irho0[2];
    T G_AB, g;
};

__device__ __forceinline__ double psi_t(double r, double ir0, int form) { return form == 1 ? r : -expm1(-r * ir0); }
__device__ __forceinline__ float psi_t(float r, float ir0, int form) { return form == 1 ? r : -expm1f(-r * ir0); }
__device__ __forceinline__ double dpsi_t(double r, double ir0, int form) { return form == 1 ? 1.0 : exp(-r * ir0) * ir0; }
__device__ __forceinline__ float dpsi_t(float r, float ir0, int form) { return form == 1 ? 1.f : expf(-r * ir0) * ir0; }

// Block accumulators: FP64, or a double-float pair (hi, lo) summed with TwoSum on the FP32 pipes.
template <typename T> struct Acc;
template <> struct Acc<double> {
    using A = double;
    __device__ static A from(double v) { return v; }
    __device__ static A add(A a, A b) { return a + b; }
    __device__ static A shfl(A a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
    __device__ static double wide(A a) { return a; }
};
template <> struct Acc<float> {
    using A = float2;
    __device__ static A from(float v) { return make_float2(v, 0.f); }
    __device__ static A add(A a, A b) { return ff_add(a, b); }
    __device__ static A shfl(A a, int o) {
        return make_float2(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o));
    }
    __device__ static double wide(A a) { return (double)a.x + (double)a.y; }
};

// Block sums of the per-thread values v[k] (k < NPAR), stored to part[blockIdx.x][k], or added
// to it (accumulate): fixed order, so results repeat bit for bit.
template <typename T>
__device__ void block_sum(const T (&v)[NPAR], typename Acc<T>::A* part, int accumulate) {
    using A = typename Acc<T>::A;
    __shared__ A red[ST / 32][NPAR];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NPAR; ++k) {
        A t = Acc<T>::from(v[k]);
        for (int o = 16; o > 0; o >>= 1) t = Acc<T>::add(t, Acc<T>::shfl(t, o));
        if (lane == 0) red[w][k] = t;
    }
    __syncthreads();
    if (threadIdx.x < NPAR) {
        A t = red[0][threadIdx.x];
        for (int i = 1; i < ST / 32; ++i) t = Acc<T>::add(t, red[i][threadIdx.x]);
        A* p = part + (long long)blockIdx.x * NPAR + threadIdx.x;
        *p = accumulate ? Acc<T>::add(*p, t) : t;
    }
}

// grad[k] += sum over the nb blocks of part[b][k]: one block, FP64, fixed order (per parameter:
// each thread's blocks in order, a butterfly over the warp, the warps in order); the eight
// parameters side by side, so their loads and reductions overlap.
template <typename T>
__global__ void __launch_bounds__(AT) k_adj_sum(const typename Acc<T>::A* __restrict__ part, long long nb,
                                                double* __restrict__ grad) {
    __shared__ double red[AT / 32][NPAR];
    double t[NPAR];
#pragma unroll
    for (int k = 0; k < NPAR; ++k) t[k] = 0.0;
    for (long long b = threadIdx.x; b < nb; b += AT)
#pragma unroll
        for (int k = 0; k < NPAR; ++k) t[k] += Acc<T>::wide(part[b * NPAR + k]);
#pragma unroll
    for (int k = 0; k < NPAR; ++k) {
        for (int o = 16; o > 0; o >>= 1) t[k] += __shfl_xor_sync(0xffffffffu, t[k], o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = t[k];
    }
    __syncthreads();
    if (threadIdx.x < NPAR) {
        double a = 0.0;
        for (int w = 0; w < AT / 32; ++w) a += red[w][threadIdx.x];
        grad[threadIdx.x] += a;
    }
}

// Intermediate fields of one adjoint step, [ns][n] each.
template <typename T>
struct AdjBuf {
    T *rho, *jx, *jz, *psi;  // the state's moments and pseudopotential
    T *qx, *qz;              // psi_s dJ/dF_s: what the force at x owes to psi_s(x + c)
    T *rx, *rz;              // rho_s dJ/dF_s: what it owes to rho_s'(x + c)
    T *dloc, *djx, *djz;     // the site's own dJ/drho_s (psi' folded in), dJ/dj_s
    T* dps;                  // psi'(rho_s)
};

// One thread per site and species (blockIdx.y = species).
template <typename T>
__global__ void __launch_bounds__(ST) k_adj_moments(const T* __restrict__ f, const AdjC<T> A, AdjBuf<T> B) {
    const long long n = (long long)A.nx * A.nz;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    {
        const int s = blockIdx.y;
        T r = 0, mx = 0, mz = 0;
#pragma unroll
        for (int l = 0; l < 9; ++l) {
            const T v = f[(s * 9 + l) * n + i];
            r += v;
            mx += v * (T)cx(l);
            mz += v * (T)cz(l);
        }
        B.rho[s * n + i] = r;
        B.jx[s * n + i] = mx;
        B.jz[s * n + i] = mz;
        B.psi[s * n + i] = psi_t(r, A.irho0[s], A.psi_form);
    }
}

template <typename T, int NS>
__global__ void __launch_bounds__(ST) k_adj_local(const T* __restrict__ f, const T* __restrict__ lam_next,
                                                  const AdjC<T> A, AdjBuf<T> B,
                                                  typename Acc<T>::A* __restrict__ part, int accumulate) {
    const long long n = (long long)A.nx * A.nz;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    T gp[NPAR] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (i < n) {
        const int z = (int)(i / A.nx), x = (int)(i - (long long)z * A.nx);
        const Nbr N(x, z, A.nx, A.nz);
        // the force at the site, keeping its three sums (attraction a, repulsion p, cross b)
        T ax[NS], az[NS], px[NS], pz[NS], bx[NS], bz[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) ax[s] = az[s] = px[s] = pz[s] = bx[s] = bz[s] = 0;
#pragma unroll
        for (int k = 0; k < 24; ++k) {
            const long long j = N.at(LKX(k), LKZ(k));
            const int q = LKX(k) * LKX(k) + LKZ(k) * LKZ(k);
            const T ex = (T)LKX(k), ez = (T)LKZ(k);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const T p = B.psi[s * n + j];
                ax[s] += A.wa[q] * p * ex;
                az[s] += A.wa[q] * p * ez;
                px[s] += A.wr[q] * p * ex;
                pz[s] += A.wr[q] * p * ez;
                if (NS == 2 && k < 8) {
                    const T ro = B.rho[(1 - s) * n + j];
                    bx[s] += A.wc[q] * ro * ex;
                    bz[s] += A.wc[q] * ro * ez;
                }
            }
        }
        T rho[NS], psi[NS], Fx[NS], Fz[NS], jx[NS], jz[NS];
        T numx = 0, numz = 0, den = 0;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            rho[s] = B.rho[s * n + i];
            psi[s] = B.psi[s * n + i];
            jx[s] = B.jx[s * n + i];
            jz[s] = B.jz[s * n + i];
            Fx[s] = -A.G1[s] * psi[s] * ax[s] - A.G2[s] * psi[s] * px[s] - A.G_AB * rho[s] * bx[s] + rho[s] * A.g;
            Fz[s] = -A.G1[s] * psi[s] * az[s] - A.G2[s] * psi[s] * pz[s] - A.G_AB * rho[s] * bz[s];
            numx += jx[s] * A.itau[s];
            numz += jz[s] * A.itau[s];
            den += rho[s] * A.itau[s];
        }
        const T iden = (T)1 / den;
        const T upx = numx * iden, upz = numz * iden;
        T dupx = 0, dupz = 0, dr[NS], dFx[NS], dFz[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const T r = rho[s], tau = A.tau[s], it = A.itau[s], ir = (T)1 / r;
            const T ux = upx + tau * Fx[s] * ir, uz = upz + tau * Fz[s] * ir;
            const T usq = ux * ux + uz * uz;
            // d/dtau of g = f - (f - feq) / tau is (f - feq) / tau^2.  sum_l (f_l - feq_l) = 0
            // (the equilibrium keeps rho), so sum_l m_l (f_l - feq_l) = sum_l (m_l - m_0)(f_l - feq_l):
            // the part of lam common to all l, often the largest, would only multiply rounding
            T ar = 0, aux = 0, auz = 0, gt = 0;
            const T m0 = lam_next[(s * 9) * n + i];
#pragma unroll
            for (int l = 0; l < 9; ++l) {
                // streaming transposed: g_l(x) became f_l(x + c_l)
                const T m = lam_next[(s * 9 + l) * n + N.at(cx(l), cz(l))];
                const T ex = (T)cx(l), ez = (T)cz(l);
                const T cu = ex * ux + ez * uz;
                const T wr = wlb<T>(l) * r;
                const T fe = wr * ((T)1 + (T)3 * cu + (T)4.5 * cu * cu - (T)1.5 * usq);
                const T dfe = m * it;  // g = f - (f - feq) / tau
                gt += (m - m0) * (f[(s * 9 + l) * n + i] - fe);
                ar += dfe * fe;
                aux += dfe * wr * ((T)3 * ex + (T)9 * cu * ex - (T)3 * ux);
                auz += dfe * wr * ((T)3 * ez + (T)9 * cu * ez - (T)3 * uz);
            }
            // u_s = u' + tau F_s / rho_s
            dupx += aux;
            dupz += auz;
            dFx[s] = aux * tau * ir;
            dFz[s] = auz * tau * ir;
            const T fu = (aux * Fx[s] + auz * Fz[s]) * ir;
            dr[s] = ar * ir - fu * tau * ir;
            gp[5 + s] += gt * it * it + fu;
        }
        // u' = sum_k j_k / tau_k / sum_k rho_k / tau_k
        const T dnx = dupx * iden, dnz = dupz * iden, dden = -(dupx * upx + dupz * upz) * iden;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const T it = A.itau[s];
            gp[5 + s] -= (jx[s] * dnx + jz[s] * dnz + rho[s] * dden) * it * it;
            dr[s] += dden * it;
            // the site's own terms of the force: F_s depends on psi_s(x), rho_s(x) and g
            const T ba = dFx[s] * ax[s] + dFz[s] * az[s], bp = dFx[s] * px[s] + dFz[s] * pz[s];
            const T bb = dFx[s] * bx[s] + dFz[s] * bz[s];
            const T dps = dpsi_t(rho[s], A.irho0[s], A.psi_form);
            gp[0 + s] -= psi[s] * ba;
            gp[2 + s] -= psi[s] * bp;
            if (NS == 2) gp[4] -= rho[s] * bb;
            gp[7] += rho[s] * dFx[s];
            B.dloc[s * n + i] = dr[s] - A.G_AB * bb + dFx[s] * A.g - dps * (A.G1[s] * ba + A.G2[s] * bp);
            B.djx[s * n + i] = dnx * it;
            B.djz[s * n + i] = dnz * it;
            B.dps[s * n + i] = dps;
            B.qx[s * n + i] = psi[s] * dFx[s];
            B.qz[s * n + i] = psi[s] * dFz[s];
            B.rx[s * n + i] = rho[s] * dFx[s];
            B.rz[s * n + i] = rho[s] * dFz[s];
        }
    }
    block_sum<T>(gp, part, accumulate);
}

// One thread per site and species (blockIdx.y = species).  f_prev (may be null): the state of the
// step before, whose moments this kernel also forms for the next adjoint step (it reads none of
// the moment fields itself, so it may overwrite them).
template <typename T, int NS>
__global__ void __launch_bounds__(ST) k_adj_final(const T* __restrict__ lam_next, const AdjC<T> A, AdjBuf<T> B,
                                                  T* __restrict__ lam, const T* __restrict__ f_prev) {
    const long long n = (long long)A.nx * A.nz;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = blockIdx.y;
    const int z = (int)(i / A.nx), x = (int)(i - (long long)z * A.nx);
    const Nbr N(x, z, A.nx, A.nz);
    // this site as the neighbour x + c of the sites x - c: their forces' dependence on its psi_s
    // and, through the cross term of the other species, on its rho_s
    const T* qx = B.qx + s * n;
    const T* qz = B.qz + s * n;
    const T* rx = B.rx + (1 - s) * n;
    const T* rz = B.rz + (1 - s) * n;
    T dps = 0, dro = 0;
#pragma unroll
    for (int k = 0; k < 24; ++k) {
        const long long jb = N.at(-LKX(k), -LKZ(k));
        const int q = LKX(k) * LKX(k) + LKZ(k) * LKZ(k);
        const T ex = (T)LKX(k), ez = (T)LKZ(k);
        dps -= (A.G1[s] * A.wa[q] + A.G2[s] * A.wr[q]) * (qx[jb] * ex + qz[jb] * ez);
        if (NS == 2 && k < 8) dro -= A.G_AB * A.wc[q] * (rx[jb] * ex + rz[jb] * ez);
    }
    const T d = B.dloc[s * n + i] + dro + B.dps[s * n + i] * dps;
    const T keep = (T)1 - A.itau[s];
    const T djx = B.djx[s * n + i], djz = B.djz[s * n + i];
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        lam[(s * 9 + l) * n + i] =
            keep * lam_next[(s * 9 + l) * n + N.at(cx(l), cz(l))] + d + djx * (T)cx(l) + djz * (T)cz(l);
    }
    if (f_prev) {
        T r = 0, mx = 0, mz = 0;
#pragma unroll
        for (int l = 0; l < 9; ++l) {
            const T v = f_prev[(s * 9 + l) * n + i];
            r += v;
            mx += v * (T)cx(l);
            mz += v * (T)cz(l);
        }
        B.rho[s * n + i] = r;
        B.jx[s * n + i] = mx;
        B.jz[s * n + i] = mz;
        B.psi[s * n + i] = psi_t(r, A.irho0[s], A.psi_form);
    }
}

// Calibration objective: J = sum_z (ubar(z) - tu(z))^2 + (rhobar_A(z) - tr(z))^2, ubar the
// x-average of u = sum_s j_x,s / sum_s rho_s, rhobar_A the x-average of rho_A.  One block per
// row forms the averages (in T, widened to FP64); k_obj_total sums the rows' shares in a fixed
// order.
template <typename T>
__global__ void __launch_bounds__(AT) k_obj_rows(const T* __restrict__ f, const AdjC<T> A, double* __restrict__ ubar,
                                                 double* __restrict__ rbar) {
    const long long n = (long long)A.nx * A.nz;
    const int z = blockIdx.x;
    T su = 0, sr = 0;
    for (int x = threadIdx.x; x < A.nx; x += AT) {
        const long long i = (long long)z * A.nx + x;
        T rt = 0, mx = 0, ra = 0;
        for (int s = 0; s < A.ns; ++s)
            for (int l = 0; l < 9; ++l) {
                const T v = f[(s * 9 + l) * n + i];
                rt += v;
                mx += v * (T)cx(l);
                if (s == 0) ra += v;
            }
        su += mx / rt;
        sr += ra;
    }
    __shared__ T red[2][AT / 32];
    for (int o = 16; o > 0; o >>= 1) {
        su += __shfl_xor_sync(0xffffffffu, su, o);
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = su;
        red[1][threadIdx.x >> 5] = sr;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < AT / 32; ++w) {
            a += (double)red[0][w];
            b += (double)red[1][w];
        }
        ubar[z] = a / A.nx;
        rbar[z] = b / A.nx;
    }
}

__global__ void __launch_bounds__(AT) k_obj_total(int nz, const double* __restrict__ tu, const double* __restrict__ tr,
                                                  const double* __restrict__ ubar, const double* __restrict__ rbar,
                                                  double* __restrict__ J) {
    __shared__ double red[AT / 32];
    double t = 0.0;
    for (int z = threadIdx.x; z < nz; z += AT)
        t += (ubar[z] - tu[z]) * (ubar[z] - tu[z]) + (rbar[z] - tr[z]) * (rbar[z] - tr[z]);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < AT / 32; ++w) a += red[w];
        *J = a;
    }
}

// dJ/df of row z: 2 (ubar - tu) / nx (c_lx - u) / rho_tot + [s = A] 2 (rhobar_A - tr) / nx; the
// row's two coefficients are formed in FP64 and rounded to T once.
template <typename T>
__global__ void __launch_bounds__(AT) k_obj_grad(const T* __restrict__ f, const AdjC<T> A, const double* __restrict__ tu,
                                                 const double* __restrict__ tr, const double* __restrict__ ubar,
                                                 const double* __restrict__ rbar, T* __restrict__ g) {
    const long long n = (long long)A.nx * A.nz;
    const int z = blockIdx.x;
    const T cu = (T)(2.0 * (ubar[z] - tu[z]) / A.nx), cr = (T)(2.0 * (rbar[z] - tr[z]) / A.nx);
    for (int x = threadIdx.x; x < A.nx; x += AT) {
        const long long i = (long long)z * A.nx + x;
        T rt = 0, mx = 0;
        for (int s = 0; s < A.ns; ++s)
            for (int l = 0; l < 9; ++l) {
                const T v = f[(s * 9 + l) * n + i];
                rt += v;
                mx += v * (T)cx(l);
            }
        const T u = mx / rt, gu = cu / rt;
        for (int s = 0; s < A.ns; ++s)
            for (int l = 0; l < 9; ++l) g[(s * 9 + l) * n + i] = gu * ((T)cx(l) - u) + (s == 0 ? cr : (T)0);
    }
}

// The initial populations are W_l rho (equilibrium at rest): dJ/drho_s = sum_l W_l lam_0.
template <typename T>
__global__ void k_adj_initial(const T* __restrict__ lam0, const AdjC<T> A, double* __restrict__ g) {
    const long long n = (long long)A.nx * A.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        for (int s = 0; s < A.ns; ++s) {
            T t = 0;
            for (int l = 0; l < 9; ++l) t += wlb<T>(l) * lam0[(s * 9 + l) * n + i];
            g[s * n + i] = (double)t;
        }
}

int grid_of(long long n) { return (int)((n + AT - 1) / AT); }

template <typename T>
AdjC<T> adj_const(const AdjConst& D) {
    AdjC<T> A;
    A.nx = D.nx;
    A.nz = D.nz;
    A.ns = D.ns;
    A.psi_form = D.psi_form;
    for (int q = 0; q < 9; ++q) {
        A.wa[q] = (T)D.wa[q];
        A.wr[q] = (T)D.wr[q];
        A.wc[q] = (T)D.wc[q];
    }
    for (int s = 0; s < 2; ++s) {
        A.G1[s] = (T)D.G1[s];
        A.G2[s] = (T)D.G2[s];
        A.tau[s] = (T)D.tau[s];
        A.itau[s] = (T)(1.0 / D.tau[s]);
        A.irho0[s] = (T)(1.0 / D.rho0[s]);
    }
    A.G_AB = (T)D.G_AB;
    A.g = (T)D.g;
    return A;
}

// Scratch of a context: the intermediate fields (12 ns n values, sized for FP64), then the block
// partials (NPAR 8-byte accumulators per block), then the objective's row averages (2 nz doubles).
size_t field_bytes(long long n, int ns) { return ((size_t)12 * ns * n * 8 + 255) & ~(size_t)255; }
int step_grid(long long n) { return (int)((n + ST - 1) / ST); }
size_t part_bytes(long long n) { return ((size_t)NPAR * step_grid(n) * 8 + 255) & ~(size_t)255; }

template <typename T>
AdjBuf<T> adj_buf(void* scratch, long long n, int ns) {
    T* p = static_cast<T*>(scratch);
    const long long m = (long long)ns * n;
    AdjBuf<T> B;
    T** fields[] = {&B.rho, &B.jx, &B.jz, &B.psi, &B.qx, &B.qz, &B.rx, &B.rz, &B.dloc, &B.djx, &B.djz, &B.dps};
    for (int k = 0; k < 12; ++k) *fields[k] = p + k * m;
    return B;
}

template <typename T, int NS>
void enqueue_steps(const AdjC<T>& A, AdjBuf<T> B, typename Acc<T>::A* part, int nb, int nsteps, const T* states,
                   long long stride, const T*& next, T* const bufs[2], cudaEvent_t* ev, cudaStream_t st) {
    for (int k = nsteps - 1, t = 0; k >= 0; --k, ++t) {
        const T* f = states + (long long)k * stride;
        T* out = bufs[t & 1];
        cudaEvent_t* e = ev ? ev + 6 * t : nullptr;
        // the moments of f: its own kernel for the first step, else formed by the previous step's
        // final kernel
        if (e) cudaEventRecord(e[0], st);
        if (t == 0) k_adj_moments<T><<<dim3(nb, NS), ST, 0, st>>>(f, A, B);
        if (e) cudaEventRecord(e[1], st), cudaEventRecord(e[2], st);
        k_adj_local<T, NS><<<nb, ST, 0, st>>>(f, next, A, B, part, t > 0);
        if (e) cudaEventRecord(e[3], st), cudaEventRecord(e[4], st);
        const T* f_prev = k > 0 ? states + (long long)(k - 1) * stride : nullptr;
        k_adj_final<T, NS><<<dim3(nb, NS), ST, 0, st>>>(next, A, B, out, f_prev);
        if (e) cudaEventRecord(e[5], st);
        next = out;
    }
}

}  // namespace

void fill_adj_const(AdjConst& A, const lbm_params& p, int nx, int nz, int ns, double body_force) {
    A.nx = nx;
    A.nz = nz;
    A.ns = ns;
    A.psi_form = p.psi_form;
    for (int q = 0; q < 9; ++q) {
        const double wa = p.weight_preset == LBM_WEIGHTS_CHEM09 ? w_belt1(q) : w_attr_paper(q);
        A.wa[q] = p.weight_norm * wa;
        A.wr[q] = p.weight_norm * w_rep(q);
        A.wc[q] = p.weight_norm * w_belt1(q);
    }
    for (int s = 0; s < 2; ++s) {
        const int ps = s < ns ? s : 0;
        A.G1[s] = p.G1[ps];
        A.G2[s] = p.G2[ps];
        A.tau[s] = p.tau[ps];
        A.rho0[s] = p.rho0[ps];
    }
    A.G_AB = ns == 2 ? p.G_AB : 0.0;
    A.g = body_force;
}

size_t adjoint_scratch_bytes(int nx, int nz, int ns) {
    const long long n = (long long)nx * nz;
    return field_bytes(n, ns) + part_bytes(n) + (size_t)2 * nz * sizeof(double);
}

template <typename T>
cudaError_t launch_adjoint_steps(const AdjConst& D, int nsteps, const T* states, long long stride, const T* lam_in,
                                 T* lam_a, T* lam_b, const T** lam_out, double* grad, void* scratch, cudaEvent_t* ev,
                                 cudaStream_t st) {
    const long long n = (long long)D.nx * D.nz;
    const AdjC<T> A = adj_const<T>(D);
    const AdjBuf<T> B = adj_buf<T>(scratch, n, D.ns);
    auto* part = reinterpret_cast<typename Acc<T>::A*>(static_cast<char*>(scratch) + field_bytes(n, D.ns));
    const int nb = step_grid(n);
    const T* next = lam_in;
    T* const bufs[2] = {lam_a, lam_b};
    if (D.ns == 2)
        enqueue_steps<T, 2>(A, B, part, nb, nsteps, states, stride, next, bufs, ev, st);
    else
        enqueue_steps<T, 1>(A, B, part, nb, nsteps, states, stride, next, bufs, ev, st);
    if (nsteps > 0) k_adj_sum<T><<<1, AT, 0, st>>>(part, nb, grad);
    *lam_out = next;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adjoint_objective(const AdjConst& D, const T* f, const double* tu, const double* tr, double* J,
                                     T* g, void* scratch, cudaStream_t st) {
    const long long n = (long long)D.nx * D.nz;
    const AdjC<T> A = adj_const<T>(D);
    double* ubar = reinterpret_cast<double*>(static_cast<char*>(scratch) + field_bytes(n, D.ns) + part_bytes(n));
    double* rbar = ubar + D.nz;
    k_obj_rows<T><<<D.nz, AT, 0, st>>>(f, A, ubar, rbar);
    k_obj_total<<<1, AT, 0, st>>>(D.nz, tu, tr, ubar, rbar, J);
    if (g) k_obj_grad<T><<<D.nz, AT, 0, st>>>(f, A, tu, tr, ubar, rbar, g);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adjoint_initial(const AdjConst& D, const T* lam0, double* g, cudaStream_t st) {
    const long long n = (long long)D.nx * D.nz;
    const AdjC<T> A = adj_const<T>(D);
    k_adj_initial<T><<<grid_of(n) < 4096 ? grid_of(n) : 4096, AT, 0, st>>>(lam0, A, g);
    return cudaGetLastError();
}

#define LBM_ADJ_INST(T)                                                                                           \
    template cudaError_t launch_adjoint_steps<T>(const AdjConst&, int, const T*, long long, const T*, T*, T*,     \
                                                 const T**, double*, void*, cudaEvent_t*, cudaStream_t);         \
    template cudaError_t launch_adjoint_objective<T>(const AdjConst&, const T*, const double*, const double*,     \
                                                     double*, T*, void*, cudaStream_t);                          \
    template cudaError_t launch_adjoint_initial<T>(const AdjConst&, const T*, double*, cudaStream_t);
LBM_ADJ_INST(double)
LBM_ADJ_INST(float)

}  // namespace lbm
