// lbm_fused.cu -- one-pass time step of the multirange Shan-Chen lattice Boltzmann model.
//
// One warp owns a strip of STRIP_W = 28 columns plus a 2-column halo on each side (the reach
// of the 5x5 stencil of Eq. FORCE) and sweeps a chunk of rows in z.  For each new row it
// reads the 9 (x species) populations of its 32 columns once from HBM (coalesced, x
// fastest), forms the density and psi, and keeps psi and rho of the last five rows in
// registers.  Two rows behind, the row is complete: the lanes gather the 5x5 psi and 3x3 rho
// neighbourhoods with warp shuffles, form the force (Eq. FORCE + cross term + body force),
// and the 28 owned lanes re-read their populations (from L1), collide (Eq. LB with the
// shifted velocity of Sec. II) and push them to their neighbours (streaming, with the
// halfway bounce-back walls of Sec. IV).  Compared with a psi pass followed by a collide
// pass this moves each population once in and once out of HBM per step.
//
// With M_OBS the same pass also accumulates the observables of the state being collided:
// per-row sums over the strip (warp reduction) and per-column sums over the chunk.
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr unsigned FULL = 0xffffffffu;

template <typename T, int NS, int MODE>
__global__ void __launch_bounds__(128) k_fused(const T* __restrict__ fin, T* __restrict__ fout,
                                               const StepConst<T> C, const SweepGeom G, const ObsPtrs O) {
    const int lane = threadIdx.x & 31;
    const int wg = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (wg >= G.nstrips * G.nchunks) return;  // whole warp
    const int strip = wg % G.nstrips;
    const int chunk = wg / G.nstrips;
    const int x = strip * STRIP_W - 2 + lane;  // column of this lane, may lie outside [0, nx)
    const int xw = wrap_index(x, C.nx);
    const bool owned = lane >= 2 && lane < 30 && x < C.nx;
    const int z0 = chunk * G.hz;
    const int z1 = min(z0 + G.hz, C.nz);
    const long long plane = C.plane;
    const int nx = C.nx, nz = C.nz, pitch = C.pitch;

    // rings: slot k holds row r - 4 + k; dr = stored density sum, ps = psi
    T dr[NS][5], ps[NS][5];
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int k = 0; k < 5; ++k) dr[s][k] = ps[s][k] = T(0);

    T acc_ps = T(0), acc_pxx = T(0);
    int bad = 0;

    for (int r = z0 - 2; r <= z1 + 1; ++r) {
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                dr[s][k] = dr[s][k + 1];
                ps[s][k] = ps[s][k + 1];
            }
        // ---- density and pseudopotential of row r (all 32 lanes) ----
        {
            const int rr = source_row(C, r);
            if (rr >= 0) {
                const T* base = fin + (long long)rr * pitch + xw;
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    T f[9];
#pragma unroll
                    for (int l = 0; l < 9; ++l) f[l] = __ldg(base + (s * 9 + l) * plane);
                    const T d = sum9(f);
                    dr[s][4] = d;
                    ps[s][4] = psi_of(C, s, C.rho_ref[s] + d);
                }
            } else {  // zero ghost row beyond a wall
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    dr[s][4] = -C.rho_ref[s];
                    ps[s][4] = T(0);
                }
            }
        }
        const int z = r - 2;
        if (z < z0) continue;  // prologue rows (warp-uniform)

        // ---- interaction at row z from the neighbourhood (all lanes take part) ----
        T F[NS][2];
        T sxx = T(0), szz = T(0), sxz = T(0);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            T p[5][5];
#pragma unroll
            for (int dz = 0; dz < 5; ++dz)
#pragma unroll
                for (int dx = -2; dx <= 2; ++dx)
                    p[dz][dx + 2] = dx == 0 ? ps[s][dz] : __shfl_sync(FULL, ps[s][dz], lane + dx);
            intra_force(C, s, p, F[s][0], F[s][1]);
            if (MODE & M_OBS) intra_stress(C, s, p, sxx, szz, sxz);
        }
        if constexpr (NS == 2) {
            T ra[3][3], rb[3][3];
#pragma unroll
            for (int dz = 0; dz < 3; ++dz)
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    const T a = dx == 0 ? dr[0][dz + 1] : __shfl_sync(FULL, dr[0][dz + 1], lane + dx);
                    const T b = dx == 0 ? dr[NS - 1][dz + 1] : __shfl_sync(FULL, dr[NS - 1][dz + 1], lane + dx);
                    ra[dz][dx + 1] = C.rho_ref[0] + a;
                    rb[dz][dx + 1] = C.rho_ref[NS - 1] + b;
                }
            cross_force(C, ra, rb, F);
            if (MODE & M_OBS) cross_stress(C, ra, rb, sxx, szz, sxz);
        }

        T rowq[NQR];
#pragma unroll
        for (int k = 0; k < NQR; ++k) rowq[k] = T(0);

        if (owned) {
            T f[NS][9], drho[NS], rho[NS];
            const T* base = fin + (long long)z * pitch + x;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
#pragma unroll
                for (int l = 0; l < 9; ++l) f[s][l] = __ldg(base + (s * 9 + l) * plane);
                drho[s] = dr[s][2];
                rho[s] = C.rho_ref[s] + drho[s];
                if (!(rho[s] > T(0)) || !(rho[s] < T(1e30))) bad = 1;
                F[s][0] += rho[s] * C.g;
            }
            if (MODE & (M_OBS | M_FIELDS)) {
                T ux, uz, pixz, rtot, mx, mz;
                site_kinetics<T, NS>(C, f, drho, rho, F, ux, uz, pixz, rtot, mx, mz);
                if (MODE & M_FIELDS) {
                    const long long i = (long long)z * nx + x;
                    const long long np = (long long)nx * nz;
#pragma unroll
                    for (int s = 0; s < NS; ++s) O.fields[s * np + i] = (double)rho[s];
                    O.fields[NS * np + i] = (double)ux;
                    O.fields[(NS + 1) * np + i] = (double)uz;
                }
                if (MODE & M_OBS) {
                    T pxx = sxx, pzz = szz;
#pragma unroll
                    for (int s = 0; s < NS; ++s) {
                        const T ir = T(1) / rho[s];
                        pxx += rho[s] * T(1.0 / 3.0) + C.kin[s] * F[s][0] * F[s][0] * ir;
                        pzz += rho[s] * T(1.0 / 3.0) + C.kin[s] * F[s][1] * F[s][1] * ir;
                    }
                    acc_ps += pxx - pzz;
                    acc_pxx += pxx;
                    rowq[QR_UX] = ux;
                    rowq[QR_RHOA] = rho[0];
                    rowq[QR_RHOB] = NS == 2 ? rho[NS - 1] : T(0);
                    rowq[QR_SXZ] = -pixz - sxz;
                    rowq[QR_MX] = mx;
                    rowq[QR_MZ] = mz;
                }
            }
            if (MODE & (M_WRITE | M_OBS)) {
                const bool wall_row = C.zbc == 1 && (z == 0 || z == nz - 1);
                if ((MODE & M_WRITE) || wall_row) {
                    collide<T, NS>(C, f, drho, rho, F);
                    // streaming: f_l(x + c_l) = g_l(x), periodic in x, periodic or walls in z
#pragma unroll
                    for (int s = 0; s < NS; ++s)
#pragma unroll
                        for (int l = 0; l < 9; ++l) {
                            int zd = z + cz(l);
                            int xd = x + cx(l);
                            xd = xd < 0 ? xd + nx : (xd >= nx ? xd - nx : xd);
                            if (C.zbc == 0) {
                                zd = zd < 0 ? zd + nz : (zd >= nz ? zd - nz : zd);
                            } else if (zd < 0 || zd >= nz) {
                                const int w = zd < 0 ? 0 : 1;
                                const T back = bounce<T>(l, f[s][l], rho[s], C.wall_u[w]);
                                if (MODE & M_WRITE) fout[(s * 9 + opp(l)) * plane + (long long)z * pitch + x] = back;
                                if (MODE & M_OBS) rowq[QR_WALLB + w] += T(cx(l)) * (f[s][l] + back);
                                continue;
                            }
                            if (MODE & M_WRITE) fout[(s * 9 + l) * plane + (long long)zd * pitch + xd] = f[s][l];
                        }
                }
            }
        }
        if (MODE & M_OBS) {
#pragma unroll
            for (int k = 0; k < NQR; ++k) {
                T v = rowq[k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
                rowq[k] = v;
            }
            if (lane == 0) {
                double* dst = O.part_row + ((long long)strip * nz + z) * NQR;
#pragma unroll
                for (int k = 0; k < NQR; ++k) dst[k] = (double)rowq[k];
            }
        }
    }
    if ((MODE & M_OBS) && owned) {
        double* dst = O.part_col + ((long long)chunk * nx + x) * NQC;
        dst[QC_PS] = (double)acc_ps;
        dst[QC_PXX] = (double)acc_pxx;
    }
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(O.flag, 1);
}

template <typename T, int NS>
cudaError_t launch_ns(int mode, const T* fin, T* fout, const StepConst<T>& C, const SweepGeom& G, const ObsPtrs& O,
                      cudaStream_t st) {
    const int warps = G.nstrips * G.nchunks;
    const dim3 block(128), grid((warps + 3) / 4);
    switch (mode) {
        case M_WRITE: k_fused<T, NS, M_WRITE><<<grid, block, 0, st>>>(fin, fout, C, G, O); break;
        case M_WRITE | M_OBS: k_fused<T, NS, M_WRITE | M_OBS><<<grid, block, 0, st>>>(fin, fout, C, G, O); break;
        case M_OBS: k_fused<T, NS, M_OBS><<<grid, block, 0, st>>>(fin, fout, C, G, O); break;
        case M_FIELDS: k_fused<T, NS, M_FIELDS><<<grid, block, 0, st>>>(fin, fout, C, G, O); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_fused(int ns, int mode, const T* fin, T* fout, const StepConst<T>& C, const SweepGeom& G,
                         const ObsPtrs& O, cudaStream_t st) {
    return ns == 1 ? launch_ns<T, 1>(mode, fin, fout, C, G, O, st) : launch_ns<T, 2>(mode, fin, fout, C, G, O, st);
}

template cudaError_t launch_fused<float>(int, int, const float*, float*, const StepConst<float>&, const SweepGeom&,
                                         const ObsPtrs&, cudaStream_t);
template cudaError_t launch_fused<double>(int, int, const double*, double*, const StepConst<double>&,
                                          const SweepGeom&, const ObsPtrs&, cudaStream_t);

}  // namespace lbm
