// lbm_adjoint.cu -- discrete adjoint of the time step (periodic lattice), in FP64.
//
// The step maps the post-streaming populations f_n to f_{n+1} = S(f_n; theta):
//   rho_s = sum_l f_l, j_s = sum_l f_l c_l (Sec. II); psi_s = psi(rho_s) (Sec. IV);
//   F_s = -psi_s(x) sum_c (G1_s w(c) + G2_s p(c)) psi_s(x + c) c            (Eq. FORCE)
//         - G_AB rho_s(x) sum_c w8(c) rho_s'(x + c) c + rho_s g x            (Sec. IV);
//   u' = sum_s j_s / tau_s / sum_s rho_s / tau_s, u_s = u' + tau_s F_s / rho_s;
//   feq_l = W_l rho_s (1 + 3 c.u_s + 9/2 (c.u_s)^2 - 3/2 u_s.u_s);
//   g_l = f_l - (f_l - feq_l) / tau_s (Eq. LB);  f_{n+1}(x + c_l, l) = g_l(x).
// Given lam_{n+1} = dJ/df_{n+1}, the kernels below form lam_n = dJ/df_n and the derivatives
// with respect to theta = (G1 A, G1 B, G2 A, G2 B, G_AB, tau A, tau B, g) by applying the
// transposed derivative of each stage in reverse order:
//   k_adj_fields   moments, psi and the force of the state f_n (the linearisation point);
//   k_adj_local    streaming transposed (a gather of lam_{n+1}), relaxation, equilibrium,
//                  shifted and common velocity: dJ/dF_s, the local dJ/drho_s, dJ/dj_s;
//   k_adj_final    the force transposed (each site gathers what its neighbours' forces owe
//                  to its psi and rho), the pseudopotential and the moments: lam_n.
// Parameter derivatives are summed per block, then over the blocks in a fixed order (FP64).
#include "lbm_consts.h"
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int AT = 256;  // threads per block

struct Site {
    int x, z;
};

__device__ __forceinline__ int wrapi(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

// (dx, dz) of the 24 interaction links, first belt first (|c|^2 = 1, 2), then 4, 5, 8
__constant__ int LKX[24] = {1, 0, -1, 0, 1, -1, -1, 1, 2, 0, -2, 0, 2, 1, -1, -2, -2, -1, 1, 2, 2, -2, -2, 2};
__constant__ int LKZ[24] = {0, 1, 0, -1, 1, 1, -1, -1, 0, 2, 0, -2, 1, 2, 2, 1, -1, -2, -2, -1, 2, 2, -2, -2};

__device__ __forceinline__ double psi_fn(const AdjConst& A, int s, double r) {
    return A.psi_form == 1 ? r : 1.0 - exp(-r / A.rho0[s]);
}
__device__ __forceinline__ double dpsi_fn(const AdjConst& A, int s, double r) {
    return A.psi_form == 1 ? 1.0 : exp(-r / A.rho0[s]) / A.rho0[s];
}

// Block sums of the per-thread values v[k] (k < K), written to part[blockIdx.x * NPAR + k0 + k].
// The parameter derivatives are summed in two fixed-order stages (blocks, then k_adj_sum), so
// a gradient does not depend on the order in which blocks finish.
constexpr int NPAR = 8;
template <int K>
__device__ void block_sum(double (&v)[K], double* part, int k0) {
    __shared__ double red[AT / 32][K];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double t = v[k];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) red[w][k] = t;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double t = 0.0;
        for (int i = 0; i < AT / 32; ++i) t += red[i][threadIdx.x];
        part[(long long)blockIdx.x * NPAR + k0 + threadIdx.x] = t;
    }
}

// grad[k] += sum over nb blocks of part[b][k]; one block, fixed order.
__global__ void __launch_bounds__(AT) k_adj_sum(const double* __restrict__ part, long long nb, double* __restrict__ grad) {
    __shared__ double red[AT / 32];
    for (int k = 0; k < NPAR; ++k) {
        double t = 0.0;
        for (long long b = threadIdx.x; b < nb; b += AT) t += part[b * NPAR + k];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0;
            for (int w = 0; w < AT / 32; ++w) a += red[w];
            grad[k] += a;
        }
        __syncthreads();
    }
}

// Moments, pseudopotential (per site), then the force (needs the neighbours' psi, rho).
__global__ void k_adj_moments(const double* __restrict__ f, const AdjConst A, double* __restrict__ rho,
                              double* __restrict__ jx, double* __restrict__ jz, double* __restrict__ psi) {
    const long long n = (long long)A.nx * A.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        for (int s = 0; s < A.ns; ++s) {
            double r = 0.0, mx = 0.0, mz = 0.0;
            for (int l = 0; l < 9; ++l) {
                const double v = f[(s * 9 + l) * n + i];
                r += v;
                mx += v * cx(l);
                mz += v * cz(l);
            }
            rho[s * n + i] = r;
            jx[s * n + i] = mx;
            jz[s * n + i] = mz;
            psi[s * n + i] = psi_fn(A, s, r);
        }
}

__global__ void k_adj_force(const AdjConst A, const double* __restrict__ rho, const double* __restrict__ psi,
                            double* __restrict__ Fx, double* __restrict__ Fz) {
    const long long n = (long long)A.nx * A.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % A.nx), z = (int)(i / A.nx);
        for (int s = 0; s < A.ns; ++s) {
            double ax = 0.0, az = 0.0, rx = 0.0, rz = 0.0, bx = 0.0, bz = 0.0;
            for (int k = 0; k < 24; ++k) {
                const long long j = (long long)wrapi(z + LKZ[k], A.nz) * A.nx + wrapi(x + LKX[k], A.nx);
                const int q = LKX[k] * LKX[k] + LKZ[k] * LKZ[k];
                const double p = psi[s * n + j];
                ax += A.wa[q] * p * LKX[k];
                az += A.wa[q] * p * LKZ[k];
                rx += A.wr[q] * p * LKX[k];
                rz += A.wr[q] * p * LKZ[k];
                if (A.ns == 2 && k < 8) {
                    const double ro = rho[(1 - s) * n + j];
                    bx += A.wc[q] * ro * LKX[k];
                    bz += A.wc[q] * ro * LKZ[k];
                }
            }
            const double ps = psi[s * n + i], r = rho[s * n + i];
            Fx[s * n + i] = -A.G1[s] * ps * ax - A.G2[s] * ps * rx - A.G_AB * r * bx + r * A.g;
            Fz[s * n + i] = -A.G1[s] * ps * az - A.G2[s] * ps * rz - A.G_AB * r * bz;
        }
    }
}

// Streaming, relaxation, equilibrium and velocities, transposed.  One site per thread.
__global__ void __launch_bounds__(AT) k_adj_local(const double* __restrict__ f, const double* __restrict__ lam_next,
                                                  const AdjConst A, const double* __restrict__ rho,
                                                  const double* __restrict__ jx, const double* __restrict__ jz,
                                                  const double* __restrict__ Fx, const double* __restrict__ Fz,
                                                  double* __restrict__ dF, double* __restrict__ drho,
                                                  double* __restrict__ djx, double* __restrict__ djz,
                                                  double* __restrict__ part) {
    const long long n = (long long)A.nx * A.nz;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double gt[2] = {0.0, 0.0};  // d/dtau A, B
    if (i < n) {
        const int x = (int)(i % A.nx), z = (int)(i / A.nx);
        double numx = 0.0, numz = 0.0, den = 0.0;
        for (int k = 0; k < A.ns; ++k) {
            numx += jx[k * n + i] / A.tau[k];
            numz += jz[k * n + i] / A.tau[k];
            den += rho[k * n + i] / A.tau[k];
        }
        const double upx = numx / den, upz = numz / den;
        double dupx = 0.0, dupz = 0.0;
        double dr[2] = {0.0, 0.0};
        for (int s = 0; s < A.ns; ++s) {
            const double r = rho[s * n + i], tau = A.tau[s];
            const double fx = Fx[s * n + i], fz = Fz[s * n + i];
            const double ux = upx + tau * fx / r, uz = upz + tau * fz / r;
            const double usq = ux * ux + uz * uz;
            double ar = 0.0, aux = 0.0, auz = 0.0;
            for (int l = 0; l < 9; ++l) {
                // streaming transposed: g_l(x) became f_l(x + c_l)
                const long long j = (long long)wrapi(z + cz(l), A.nz) * A.nx + wrapi(x + cx(l), A.nx);
                const double m = lam_next[(s * 9 + l) * n + j];
                const double cu = cx(l) * ux + cz(l) * uz;
                const double fe = wlb<double>(l) * r * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
                const double dfe = m / tau;  // g = f - (f - feq) / tau
                gt[s] += m * (f[(s * 9 + l) * n + i] - fe) / (tau * tau);
                ar += dfe * fe / r;
                aux += dfe * wlb<double>(l) * r * (3.0 * cx(l) + 9.0 * cu * cx(l) - 3.0 * ux);
                auz += dfe * wlb<double>(l) * r * (3.0 * cz(l) + 9.0 * cu * cz(l) - 3.0 * uz);
            }
            // u_s = u' + tau F_s / rho_s
            dupx += aux;
            dupz += auz;
            dF[(s * 2 + 0) * n + i] = aux * tau / r;
            dF[(s * 2 + 1) * n + i] = auz * tau / r;
            dr[s] += ar - (aux * fx + auz * fz) * tau / (r * r);
            gt[s] += (aux * fx + auz * fz) / r;
        }
        // u' = sum_k j_k / tau_k / sum_k rho_k / tau_k
        const double dnx = dupx / den, dnz = dupz / den, dden = -(dupx * upx + dupz * upz) / den;
        for (int k = 0; k < A.ns; ++k) {
            const double tk = A.tau[k];
            djx[k * n + i] = dnx / tk;
            djz[k * n + i] = dnz / tk;
            drho[k * n + i] = dr[k] + dden / tk;
            gt[k] += -(jx[k * n + i] * dnx + jz[k * n + i] * dnz + rho[k * n + i] * dden) / (tk * tk);
        }
    }
    block_sum<2>(gt, part, 5);
}

// The force transposed (gathered from the neighbours whose force used this site), then the
// pseudopotential and the moments: lam_n.
__global__ void __launch_bounds__(AT) k_adj_final(const double* __restrict__ lam_next, const AdjConst A,
                                                  const double* __restrict__ rho, const double* __restrict__ psi,
                                                  const double* __restrict__ dF, const double* __restrict__ drho,
                                                  const double* __restrict__ djx, const double* __restrict__ djz,
                                                  double* __restrict__ lam, double* __restrict__ part) {
    const long long n = (long long)A.nx * A.nz;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double gp[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};  // G1 A, B; G2 A, B; G_AB; g
    if (i < n) {
        const int x = (int)(i % A.nx), z = (int)(i / A.nx);
        double dps[2] = {0.0, 0.0}, dro[2] = {0.0, 0.0};
        for (int s = 0; s < A.ns; ++s) {
            dro[s] += drho[s * n + i];
            const double bx = dF[(s * 2 + 0) * n + i], bz = dF[(s * 2 + 1) * n + i];
            const double ps = psi[s * n + i], r = rho[s * n + i];
            double ax = 0.0, az = 0.0, rx = 0.0, rz = 0.0, cxs = 0.0, czs = 0.0;
            for (int k = 0; k < 24; ++k) {
                const int q = LKX[k] * LKX[k] + LKZ[k] * LKZ[k];
                // this site as the source of the force: its neighbours' psi and rho
                const long long jf = (long long)wrapi(z + LKZ[k], A.nz) * A.nx + wrapi(x + LKX[k], A.nx);
                const double pf = psi[s * n + jf];
                ax += A.wa[q] * pf * LKX[k];
                az += A.wa[q] * pf * LKZ[k];
                rx += A.wr[q] * pf * LKX[k];
                rz += A.wr[q] * pf * LKZ[k];
                // this site as a neighbour of x - c: what that site's force owes to its psi
                const long long jb = (long long)wrapi(z - LKZ[k], A.nz) * A.nx + wrapi(x - LKX[k], A.nx);
                const double bbc = dF[(s * 2 + 0) * n + jb] * LKX[k] + dF[(s * 2 + 1) * n + jb] * LKZ[k];
                dps[s] += -psi[s * n + jb] * (A.G1[s] * A.wa[q] + A.G2[s] * A.wr[q]) * bbc;
                if (A.ns == 2 && k < 8) {
                    cxs += A.wc[q] * rho[(1 - s) * n + jf] * LKX[k];
                    czs += A.wc[q] * rho[(1 - s) * n + jf] * LKZ[k];
                    // the other species' force at x - c used this site's rho_s as its rho_s'
                    const double obc = dF[((1 - s) * 2 + 0) * n + jb] * LKX[k] + dF[((1 - s) * 2 + 1) * n + jb] * LKZ[k];
                    dro[s] += -A.G_AB * rho[(1 - s) * n + jb] * A.wc[q] * obc;
                }
            }
            dps[s] += -(A.G1[s] * (bx * ax + bz * az) + A.G2[s] * (bx * rx + bz * rz));
            gp[0 + s] += -ps * (bx * ax + bz * az);
            gp[2 + s] += -ps * (bx * rx + bz * rz);
            if (A.ns == 2) {
                dro[s] += -A.G_AB * (bx * cxs + bz * czs);
                gp[4] += -r * (bx * cxs + bz * czs);
            }
            dro[s] += bx * A.g;
            gp[5] += r * bx;
        }
        for (int s = 0; s < A.ns; ++s) {
            const double d = dro[s] + dpsi_fn(A, s, rho[s * n + i]) * dps[s];
            const double keep = 1.0 - 1.0 / A.tau[s];
            for (int l = 0; l < 9; ++l) {
                const long long j = (long long)wrapi(z + cz(l), A.nz) * A.nx + wrapi(x + cx(l), A.nx);
                lam[(s * 9 + l) * n + i] =
                    keep * lam_next[(s * 9 + l) * n + j] + d + djx[s * n + i] * cx(l) + djz[s * n + i] * cz(l);
            }
        }
    }
    double g5[5] = {gp[0], gp[1], gp[2], gp[3], gp[4]};
    block_sum<5>(g5, part, 0);
    double g1[1] = {gp[5]};
    block_sum<1>(g1, part, 7);
}

// Calibration objective: J = sum_z (ubar(z) - tu(z))^2 + (rhobar_A(z) - tr(z))^2, ubar the
// x-average of u = sum_s j_x,s / sum_s rho_s, rhobar_A the x-average of rho_A.  One block per
// row forms the averages; k_obj_total sums the rows' shares in a fixed order.
__global__ void __launch_bounds__(AT) k_obj_rows(const double* __restrict__ f, const AdjConst A,
                                                 double* __restrict__ ubar, double* __restrict__ rbar) {
    const long long n = (long long)A.nx * A.nz;
    const int z = blockIdx.x;
    double su = 0.0, sr = 0.0;
    for (int x = threadIdx.x; x < A.nx; x += AT) {
        const long long i = (long long)z * A.nx + x;
        double rt = 0.0, mx = 0.0, ra = 0.0;
        for (int s = 0; s < A.ns; ++s)
            for (int l = 0; l < 9; ++l) {
                const double v = f[(s * 9 + l) * n + i];
                rt += v;
                mx += v * cx(l);
                if (s == 0) ra += v;
            }
        su += mx / rt;
        sr += ra;
    }
    __shared__ double red[2][AT / 32];
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
            a += red[0][w];
            b += red[1][w];
        }
        ubar[z] = a / A.nx;
        rbar[z] = b / A.nx;
    }
}

__global__ void __launch_bounds__(AT) k_obj_total(const AdjConst A, const double* __restrict__ tu,
                                                  const double* __restrict__ tr, const double* __restrict__ ubar,
                                                  const double* __restrict__ rbar, double* __restrict__ J) {
    __shared__ double red[AT / 32];
    double t = 0.0;
    for (int z = threadIdx.x; z < A.nz; z += AT)
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

__global__ void k_obj_grad(const double* __restrict__ f, const AdjConst A, const double* __restrict__ tu,
                           const double* __restrict__ tr, const double* __restrict__ ubar,
                           const double* __restrict__ rbar, double* __restrict__ g) {
    const long long n = (long long)A.nx * A.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(i / A.nx);
        double rt = 0.0, mx = 0.0;
        for (int s = 0; s < A.ns; ++s)
            for (int l = 0; l < 9; ++l) {
                const double v = f[(s * 9 + l) * n + i];
                rt += v;
                mx += v * cx(l);
            }
        const double u = mx / rt;
        const double gu = 2.0 * (ubar[z] - tu[z]) / A.nx / rt, gr = 2.0 * (rbar[z] - tr[z]) / A.nx;
        for (int s = 0; s < A.ns; ++s)
            for (int l = 0; l < 9; ++l) g[(s * 9 + l) * n + i] = gu * (cx(l) - u) + (s == 0 ? gr : 0.0);
    }
}

// The initial populations are W_l rho (equilibrium at rest): dJ/drho_s = sum_l W_l lam_0.
__global__ void k_adj_initial(const double* __restrict__ lam0, const AdjConst A, double* __restrict__ g) {
    const long long n = (long long)A.nx * A.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        for (int s = 0; s < A.ns; ++s) {
            double t = 0.0;
            for (int l = 0; l < 9; ++l) t += wlb<double>(l) * lam0[(s * 9 + l) * n + i];
            g[s * n + i] = t;
        }
}

int grid_of(long long n) { return (int)((n + AT - 1) / AT); }

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

cudaError_t launch_adjoint_step(const AdjConst& A, const double* f, const double* lam_next, double* lam,
                                double* grad, double* scratch, cudaStream_t st) {
    const long long n = (long long)A.nx * A.nz;
    const long long m = (long long)A.ns * n;
    double *rho = scratch, *jx = rho + m, *jz = jx + m, *psi = jz + m, *Fx = psi + m, *Fz = Fx + m;
    double *dF = Fz + m, *drho = dF + 2 * m, *djx = drho + m, *djz = djx + m, *part = djz + m;
    const int gb = grid_of(n) < 4096 ? grid_of(n) : 4096;
    k_adj_moments<<<gb, AT, 0, st>>>(f, A, rho, jx, jz, psi);
    k_adj_force<<<gb, AT, 0, st>>>(A, rho, psi, Fx, Fz);
    k_adj_local<<<grid_of(n), AT, 0, st>>>(f, lam_next, A, rho, jx, jz, Fx, Fz, dF, drho, djx, djz, part);
    k_adj_final<<<grid_of(n), AT, 0, st>>>(lam_next, A, rho, psi, dF, drho, djx, djz, lam, part);
    k_adj_sum<<<1, AT, 0, st>>>(part, grid_of(n), grad);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_objective(const AdjConst& A, const double* f, const double* tu, const double* tr,
                                     double* J, double* g, double* scratch, cudaStream_t st) {
    const long long n = (long long)A.nx * A.nz;
    double *ubar = scratch, *rbar = scratch + A.nz;
    k_obj_rows<<<A.nz, AT, 0, st>>>(f, A, ubar, rbar);
    k_obj_total<<<1, AT, 0, st>>>(A, tu, tr, ubar, rbar, J);
    if (g) k_obj_grad<<<grid_of(n) < 4096 ? grid_of(n) : 4096, AT, 0, st>>>(f, A, tu, tr, ubar, rbar, g);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_initial(const AdjConst& A, const double* lam0, double* g, cudaStream_t st) {
    const long long n = (long long)A.nx * A.nz;
    k_adj_initial<<<grid_of(n) < 4096 ? grid_of(n) : 4096, AT, 0, st>>>(lam0, A, g);
    return cudaGetLastError();
}

long long adjoint_scratch_doubles(int nx, int nz, int ns) {
    const long long n = (long long)nx * nz;
    const long long step = 11LL * ns * n + (long long)NPAR * grid_of(n);
    return step > 2LL * nz ? step : 2LL * nz;
}

}  // namespace lbm
