// lbm_tile.cu -- one-pass time step on 2-D tiles with the density halo recomputed.
//
// A block owns a TPX x TPZ tile of sites (one warp per tile row).  Phase A forms rho and psi of
// the (TPX + 4) x (TPZ + 4) neighbourhood of the tile into shared memory: every thread does its
// own site (keeping its 9 x NS populations in registers) and the 2-cell halo ring is shared out
// over the block.  With the push layout (the stored state is post-streaming) the density of a
// site needs only that site's populations, so the halo costs a re-read of neighbouring tiles'
// populations, which their own blocks are reading at the same time (L2 hits), and no extra
// pass over HBM.  Phase B gathers the 5 x 5 psi and 3 x 3 rho neighbourhoods from shared
// memory, forms the force (Eq. FORCE + cross term + body force), collides (Eq. LB with the
// shifted velocity of Sec. II) and pushes (streaming with the walls of Sec. IV); with M_OBS it
// also forms the observables' partial sums (per tile row and per tile column).
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int HW = TPX + 4;  // halo tile width

// TZ: tile height (8 or 16 rows, one warp per row).  Registers are capped so that 32 warps fit
// on an SM in FP32 (64 per thread); FP64 keeps more registers and half the warps.
template <typename T, int NS, int MODE, int TZ>
__global__ void __launch_bounds__(TPX* TZ, (sizeof(T) == 4 ? 1024 : 512) / (TPX * TZ))
    k_tile(const T* __restrict__ fin, T* __restrict__ fout, const StepConst<T> C, const ObsPtrs O, int nxpart,
           int nzpart) {
    constexpr int TPZ = TZ;
    constexpr int HH = TPZ + 4;  // halo tile height
    constexpr int NRING = HW * HH - TPX * TPZ;
    __shared__ T sps[NS][HH][HW];
    __shared__ T srh[NS][HH][HW];
    __shared__ T colsum[TPZ][NQC][TPX];
    const int tx = threadIdx.x, tz = threadIdx.y, tid = tz * TPX + tx;
    const int x0 = blockIdx.x * TPX, z0 = blockIdx.y * TPZ;
    const int x = x0 + tx, z = z0 + tz;
    const int nx = C.nx, nz = C.nz;
    const long long plane = C.plane;
    const bool live = x < nx && z < nz;

    // ---- phase A: densities and psi of the tile and its 2-cell ring ----
    // Every thread loads its own site and (threads below NRING) one ring site before summing,
    // so both sets of loads are in flight together.
    T f[NS][9];
    T drho[NS];
    int rhx = 0, rhz = 0;
    const bool ring = tid < NRING;
    if (ring) {  // ring order: top two rows, bottom two rows, then two columns on each side
        if (tid < 2 * HW) {
            rhz = tid / HW;
            rhx = tid % HW;
        } else if (tid < 4 * HW) {
            rhz = HH - 2 + (tid - 2 * HW) / HW;
            rhx = (tid - 2 * HW) % HW;
        } else {
            const int j = tid - 4 * HW;  // 0 .. 4 TPZ - 1
            rhz = 2 + (j >> 2);
            const int c = j & 3;
            rhx = c < 2 ? c : HW - 4 + c;
        }
    }
    static_assert(NRING <= TPX * TPZ, "one ring site per thread at most");
    const int own_x = live ? x : x0 - 2 + (tx + 2), own_z = live ? z : z0 - 2 + (tz + 2);
    const int own_r = source_row(C, own_z);
    const int ring_r = ring ? source_row(C, z0 - 2 + rhz) : -1;
    auto wrapx = [&](int xs) {
        const int xw = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
        return (xw >= 0 && xw < nx) ? xw : wrap_index(xs, nx);
    };
    T g[NS][9];
    if (own_r >= 0) {
        const T* base = fin + (long long)own_r * C.pitch + wrapx(own_x);
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int l = 0; l < 9; ++l) f[s][l] = __ldg(base + (s * 9 + l) * plane);
    }
    if (ring_r >= 0) {
        const T* base = fin + (long long)ring_r * C.pitch + wrapx(x0 - 2 + rhx);
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int l = 0; l < 9; ++l) g[s][l] = __ldg(base + (s * 9 + l) * plane);
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        drho[s] = own_r >= 0 ? sum9(f[s]) : -C.rho_ref[s];
        const T r = C.rho_ref[s] + drho[s];
        srh[s][tz + 2][tx + 2] = r;
        sps[s][tz + 2][tx + 2] = own_r >= 0 ? psi_of(C, s, r) : T(0);
        if (ring) {
            const T rr = ring_r >= 0 ? C.rho_ref[s] + sum9(g[s]) : T(0);
            srh[s][rhz][rhx] = rr;
            sps[s][rhz][rhx] = ring_r >= 0 ? psi_of(C, s, rr) : T(0);
        }
    }
    __syncthreads();

    // ---- phase B: interaction, collision, streaming, observables ----
    T F[NS][2];
    T sxx = T(0), szz = T(0), sxz = T(0);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        T p[5][5];
#pragma unroll
        for (int dz = 0; dz < 5; ++dz)
#pragma unroll
            for (int dx = 0; dx < 5; ++dx) p[dz][dx] = sps[s][tz + dz][tx + dx];
        intra_force(C, s, p, F[s][0], F[s][1]);
        if (MODE & M_OBS) intra_stress(C, s, p, sxx, szz, sxz);
    }
    if constexpr (NS == 2) {
        T ra[3][3], rb[3][3];
#pragma unroll
        for (int dz = 0; dz < 3; ++dz)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                ra[dz][dx] = srh[0][tz + 1 + dz][tx + 1 + dx];
                rb[dz][dx] = srh[1][tz + 1 + dz][tx + 1 + dx];
            }
        cross_force(C, ra, rb, F);
        if (MODE & M_OBS) cross_stress(C, ra, rb, sxx, szz, sxz);
    }

    T rowq[NQR];
#pragma unroll
    for (int k = 0; k < NQR; ++k) rowq[k] = T(0);
    T cps = T(0), cpx = T(0);
    int bad = 0;
    if (live) {
        T rho[NS], ir[NS], jx[NS], jz[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            rho[s] = C.rho_ref[s] + drho[s];
            if (!(rho[s] > T(0)) || !(rho[s] < T(1e30))) bad = 1;
            ir[s] = div_(T(1), rho[s]);
            momentum9(f[s], jx[s], jz[s]);
            F[s][0] += rho[s] * C.g;
        }
        if (MODE & (M_OBS | M_FIELDS)) {
            T ux, uz, pixz, rtot, mx, mz;
            site_kinetics<T, NS>(C, f, rho, ir, jx, jz, F, ux, uz, pixz, rtot, mx, mz);
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
                    pxx += rho[s] * T(1.0 / 3.0) + C.kin[s] * F[s][0] * F[s][0] * ir[s];
                    pzz += rho[s] * T(1.0 / 3.0) + C.kin[s] * F[s][1] * F[s][1] * ir[s];
                }
                cps = pxx - pzz;
                cpx = pxx;
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
                collide<T, NS>(C, f, drho, rho, ir, jx, jz, F);
                const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
                const long long rz0 = (long long)z * C.pitch;
                const long long rzm = (long long)(z == 0 ? nz - 1 : z - 1) * C.pitch;
                const long long rzp = (long long)(z == nz - 1 ? 0 : z + 1) * C.pitch;
                if (!wall_row) {  // warp-uniform: every destination lies in the lattice
                    if (MODE & M_WRITE) {
#pragma unroll
                        for (int s = 0; s < NS; ++s)
#pragma unroll
                            for (int l = 0; l < 9; ++l) {
                                const long long row = cz(l) < 0 ? rzm : (cz(l) > 0 ? rzp : rz0);
                                const int col = cx(l) < 0 ? xm : (cx(l) > 0 ? xp : x);
                                fout[(s * 9 + l) * plane + row + col] = f[s][l];
                            }
                    }
                } else {
#pragma unroll
                    for (int s = 0; s < NS; ++s)
#pragma unroll
                        for (int l = 0; l < 9; ++l) {
                            const int zd = z + cz(l);
                            const int col = cx(l) < 0 ? xm : (cx(l) > 0 ? xp : x);
                            if (zd < 0 || zd >= nz) {  // halfway bounce-back with Ladd's term
                                const int w = zd < 0 ? 0 : 1;
                                const T back = bounce<T>(l, f[s][l], rho[s], C.wall_u[w]);
                                if (MODE & M_WRITE) fout[(s * 9 + opp(l)) * plane + rz0 + x] = back;
                                if (MODE & M_OBS) {
                                    const T dm = T(cx(l)) * (f[s][l] + back);
                                    if (w == 0)
                                        rowq[QR_WALLB] += dm;
                                    else
                                        rowq[QR_WALLT] += dm;
                                }
                            } else if (MODE & M_WRITE) {
                                fout[(s * 9 + l) * plane + (long long)zd * C.pitch + col] = f[s][l];
                            }
                        }
                }
            }
        }
    }
    if (__any_sync(FULL, bad) && tx == 0) atomicOr(O.flag, 1);
    if (MODE & M_OBS) {
        // per-row sums over the 32 sites of this warp: transpose-reduce, lane 4q holds quantity q
        static_assert(NQR == 8, "row reduction is written for 8 quantities");
        T v4[4], v2[2], v1;
        const bool b4 = tx & 16, b3 = tx & 8, b2 = tx & 4;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const T keep = b4 ? rowq[k + 4] : rowq[k], send = b4 ? rowq[k] : rowq[k + 4];
            v4[k] = keep + __shfl_xor_sync(FULL, send, 16);
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const T keep = b3 ? v4[k + 2] : v4[k], send = b3 ? v4[k] : v4[k + 2];
            v2[k] = keep + __shfl_xor_sync(FULL, send, 8);
        }
        {
            const T keep = b2 ? v2[1] : v2[0], send = b2 ? v2[0] : v2[1];
            v1 = keep + __shfl_xor_sync(FULL, send, 4);
        }
        v1 += __shfl_xor_sync(FULL, v1, 2);
        v1 += __shfl_xor_sync(FULL, v1, 1);
        if ((tx & 3) == 0 && z < nz) {
            const int q = (b4 ? 4 : 0) + (b3 ? 2 : 0) + (b2 ? 1 : 0);
            static_cast<T*>(O.part_row)[((long long)z * nxpart + blockIdx.x) * NQR + q] = v1;
        }
        // per-column sums over the TPZ rows of the tile
        colsum[tz][QC_PS][tx] = cps;
        colsum[tz][QC_PXX][tx] = cpx;
        __syncthreads();
        if (tz < NQC && x < nx) {
            T v = T(0);
#pragma unroll
            for (int r = 0; r < TPZ; ++r) v += colsum[r][tz][tx];
            static_cast<T*>(O.part_col)[((long long)x * nzpart + blockIdx.y) * NQC + tz] = v;
        }
    }
}

template <typename T, int NS, int MODE, int TZ>
cudaError_t launch_mode(const T* fin, T* fout, const StepConst<T>& C, const ObsPtrs& O, cudaStream_t st) {
    const int nxpart = (C.nx + TPX - 1) / TPX, nzpart = (C.nz + TZ - 1) / TZ;
    const dim3 block(TPX, TZ), grid(nxpart, nzpart);
    k_tile<T, NS, MODE, TZ><<<grid, block, 0, st>>>(fin, fout, C, O, nxpart, nzpart);
    return cudaGetLastError();
}

template <typename T, int NS, int TZ>
cudaError_t launch_ns(int mode, const T* fin, T* fout, const StepConst<T>& C, const ObsPtrs& O, cudaStream_t st) {
    switch (mode) {
        case M_WRITE: return launch_mode<T, NS, M_WRITE, TZ>(fin, fout, C, O, st);
        case M_WRITE | M_OBS: return launch_mode<T, NS, M_WRITE | M_OBS, TZ>(fin, fout, C, O, st);
        case M_OBS: return launch_mode<T, NS, M_OBS, TZ>(fin, fout, C, O, st);
        case M_FIELDS: return launch_mode<T, NS, M_FIELDS, TZ>(fin, fout, C, O, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_tile(int ns, int mode, int tile_rows, const T* fin, T* fout, const StepConst<T>& C,
                        const ObsPtrs& O, cudaStream_t st) {
    if (tile_rows == 16)
        return ns == 1 ? launch_ns<T, 1, 16>(mode, fin, fout, C, O, st) : launch_ns<T, 2, 16>(mode, fin, fout, C, O, st);
    if (tile_rows == 8)
        return ns == 1 ? launch_ns<T, 1, 8>(mode, fin, fout, C, O, st) : launch_ns<T, 2, 8>(mode, fin, fout, C, O, st);
    return cudaErrorInvalidValue;
}

template cudaError_t launch_tile<float>(int, int, int, const float*, float*, const StepConst<float>&, const ObsPtrs&,
                                        cudaStream_t);
template cudaError_t launch_tile<double>(int, int, int, const double*, double*, const StepConst<double>&,
                                         const ObsPtrs&, cudaStream_t);

}  // namespace lbm
