// lbm_obs.cu -- initial state, state export and the FP64 reduction of the observables.
#include "lbm_internal.h"

namespace lbm {

namespace {

// Populations at the equilibrium of Sec. II for given rho, u (stored as deviations from
// W_l rho_ref; rho_ref = 0 stores plain values).  The arithmetic is done in FP64.
template <typename T>
__global__ void k_init(int ns, T* __restrict__ f, const double* __restrict__ rho, const double* __restrict__ u,
                       const StepConst<T> C) {
    const long long n = (long long)C.nx * C.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % C.nx), z = (int)(i / C.nx);
        const double ux = u ? u[i] : 0.0, uz = u ? u[n + i] : 0.0;
        for (int s = 0; s < ns; ++s) {
            const double r = rho[s * n + i];
            const double dr = r - (double)C.rho_ref[s];
            for (int l = 0; l < 9; ++l)
                f[(s * 9 + l) * C.plane + (long long)z * C.pitch + x] = (T)feq_dev<double>(l, dr, r, ux, uz);
        }
    }
}

template <typename T>
__global__ void k_export(int ns, const T* __restrict__ f, double* __restrict__ out, const StepConst<T> C) {
    const long long n = (long long)C.nx * C.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % C.nx), z = (int)(i / C.nx);
        for (int s = 0; s < ns; ++s)
            for (int l = 0; l < 9; ++l)
                out[(s * 9 + l) * n + i] = (double)f[(s * 9 + l) * C.plane + (long long)z * C.pitch + x] +
                                           wlb<double>(l) * (double)C.rho_ref[s];
    }
}

constexpr int RB_THREADS = 256;
constexpr int NSC = 5;  // scalar slots per row / column: mass A, mass B, momentum x, z; gamma

template <typename PT>
__device__ PT warp_sum(PT v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Phase 1, one warp per row: the row's sums over its column groups, its profile entries
// (x-averages), the fluidity of Eq. fluidity (shear rate = central difference of ux_z,
// one-sided at wall rows, wrapped when periodic) and, when sampling, the row's time sums.  One
// warp per column: the z-averages of P_xx - P_zz and P_xx.  Phase 2 (the last block to
// finish): the global scalars (mass, momentum, gamma, wall stress) summed in FP64.
// Group sums within a row or a column stay in the populations' precision PT (in FP32 mode they
// are sums of FP32 values; FP64 arithmetic is scarce on this GPU); each row or column total is
// widened to FP64 once.  All sums run in a fixed order, so results are repeatable.
template <typename PT>
__global__ void __launch_bounds__(RB_THREADS) k_reduce(const ObsPtrs O, int nxpart, int nzpart, int nx, int nz, int zbc,
                                                       int nrowblocks, double* __restrict__ row_sum,
                                                       double* __restrict__ col_sum, unsigned* ticket,
                                                       double* __restrict__ out, double* __restrict__ avg,
                                                       int accumulate, double inx, double inz) {
    __shared__ double sh5[NSC * RB_THREADS];
    __shared__ bool last;
    constexpr int WPB = RB_THREADS / 32;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const PT* const prow = static_cast<const PT*>(O.part_row);
    const PT* const pcol = static_cast<const PT*>(O.part_col);
    double* const ux = out + O_PROF;
    double* const rz = ux + nz;
    double* const sx = rz + 2LL * nz;
    double* const fl = sx + nz;
    double* const ps = fl + nz;
    double* const px = ps + nx;
    if ((int)blockIdx.x < nrowblocks) {
        const int z = blockIdx.x * WPB + warp;
        if (z < nz) {
            int zl = z - 1, zr = z + 1;
            double wl = 0.5, wr = 0.5;
            if (nz == 1) {
                zl = zr = z;
            } else if (zbc == 0) {
                zl = z == 0 ? nz - 1 : z - 1;
                zr = z == nz - 1 ? 0 : z + 1;
            } else if (z == 0) {
                zl = 0;
                wl = wr = 1.0;
            } else if (z == nz - 1) {
                zr = nz - 1;
                wl = wr = 1.0;
            }
            PT v[NQR + 2];
#pragma unroll
            for (int k = 0; k < NQR + 2; ++k) v[k] = PT(0);
            for (int p = lane; p < nxpart; p += 32) {
                const PT* src = prow + ((long long)z * nxpart + p) * NQR;
#pragma unroll
                for (int k = 0; k < NQR; ++k) v[k] += src[k];
                v[NQR] += prow[((long long)zl * nxpart + p) * NQR + QR_UX];
                v[NQR + 1] += prow[((long long)zr * nxpart + p) * NQR + QR_UX];
            }
#pragma unroll
            for (int k = 0; k < NQR + 2; ++k) v[k] = warp_sum(v[k]);
            if (lane == 0) {
                // this row's contributions to the scalars (mass A, mass B, momentum x, z)
                double* w = col_sum + (long long)z * NSC;
                w[0] = (double)v[QR_RHOA];
                w[1] = (double)v[QR_RHOB];
                w[2] = (double)v[QR_MX];
                w[3] = (double)v[QR_MZ];
                if (z == 0) row_sum[0] = (double)v[QR_WALLB];
                if (z == nz - 1) row_sum[1] = (double)v[QR_WALLT];
                const double gd = nz == 1 ? 0.0 : (wr * (double)v[NQR + 1] - wl * (double)v[NQR]) * inx;
                const double sxz = (double)v[QR_SXZ] * inx;
                ux[z] = (double)v[QR_UX] * inx;
                rz[z] = (double)v[QR_RHOA] * inx;
                rz[nz + z] = (double)v[QR_RHOB] * inx;
                sx[z] = sxz;
                fl[z] = gd / sxz;
                if (accumulate) {
                    double* a = avg + O_PROF;
                    a[z] += ux[z];
                    a[nz + z] += rz[z];
                    a[2LL * nz + z] += rz[nz + z];
                    a[3LL * nz + z] += sxz;
                    a[4LL * nz + z] += fl[z];
                }
            }
        }
    } else {
        const int x = (blockIdx.x - nrowblocks) * WPB + warp;
        if (x < nx) {
            PT v[NQC];
#pragma unroll
            for (int k = 0; k < NQC; ++k) v[k] = PT(0);
            for (int p = lane; p < nzpart; p += 32) {
                const PT* src = pcol + ((long long)x * nzpart + p) * NQC;
#pragma unroll
                for (int k = 0; k < NQC; ++k) v[k] += src[k];
            }
#pragma unroll
            for (int k = 0; k < NQC; ++k) v[k] = warp_sum(v[k]);
            if (lane == 0) {
                ps[x] = (double)v[QC_PS] * inz;
                px[x] = (double)v[QC_PXX] * inz;
                col_sum[((long long)nz + x) * NSC + 4] = ps[x];  // this column's share of gamma
                if (accumulate) {
                    double* a = avg + O_PROF + 5LL * nz;
                    a[x] += ps[x];
                    a[nx + x] += px[x];
                }
            }
        }
    }
    // the block's writes happen before thread 0's fence (barrier), and the fence is cumulative:
    // whichever block draws the last ticket sees every block's results
    __syncthreads();
    if (t == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
        if (last) __threadfence();
    }
    __syncthreads();
    if (!last) return;

    // scalars: rows hold slots 0..3, columns slot 4, in fixed order
    double acc[NSC] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int z = t; z < nz; z += RB_THREADS)
        for (int k = 0; k < 4; ++k) acc[k] += col_sum[(long long)z * NSC + k];
    for (int x = t; x < nx; x += RB_THREADS) acc[4] += col_sum[((long long)nz + x) * NSC + 4];
    double* shv = sh5;
    for (int k = 0; k < NSC; ++k) shv[k * RB_THREADS + t] = acc[k];
    __syncthreads();
    for (int o = RB_THREADS / 2; o > 0; o >>= 1) {
        if (t < o)
            for (int k = 0; k < NSC; ++k) shv[k * RB_THREADS + t] += shv[k * RB_THREADS + t + o];
        __syncthreads();
    }
    if (t == 0) {
        const double m0 = shv[0], m1 = shv[RB_THREADS], mx = shv[2 * RB_THREADS], mz = shv[3 * RB_THREADS],
                     g = shv[4 * RB_THREADS];
        out[O_MASS] = m0;
        out[O_MASS + 1] = m1;
        out[O_MOM] = mx;
        out[O_MOM + 1] = mz;
        out[O_GAMMA] = g;
        out[O_WALL] = zbc ? row_sum[0] * inx : 0.0;
        out[O_WALL + 1] = zbc ? row_sum[1] * inx : 0.0;
        const bool bad = (O.flag[0] & 1) || !isfinite(m0) || !isfinite(m1) || !isfinite(mx) || !isfinite(mz) ||
                         !isfinite(g);
        out[O_BAD] = bad ? 1.0 : 0.0;
        if (accumulate) {
            for (int i = 0; i < O_BAD; ++i) avg[i] += out[i];
            avg[O_BAD] = (avg[O_BAD] != 0.0 || bad) ? 1.0 : 0.0;
            avg[O_COUNT] += 1.0;
        }
        *ticket = 0u;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_init(int ns, T* f, const double* rho, const double* u, const StepConst<T>& C, cudaStream_t st) {
    const long long n = (long long)C.nx * C.nz;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_init<T><<<blocks, 256, 0, st>>>(ns, f, rho, u, C);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_export(int ns, const T* f, double* out, const StepConst<T>& C, cudaStream_t st) {
    const long long n = (long long)C.nx * C.nz;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_export<T><<<blocks, 256, 0, st>>>(ns, f, out, C);
    return cudaGetLastError();
}

cudaError_t launch_reduce(int precision_bytes, const ObsPtrs& O, int nxpart, int nzpart, int nx, int nz, int zbc,
                          double* row_sum, double* col_sum, unsigned* ticket, double* out, double* avg,
                          int accumulate, cudaStream_t st) {
    const int rb = (nz + RB_THREADS / 32 - 1) / (RB_THREADS / 32);
    const int cb = (nx + RB_THREADS / 32 - 1) / (RB_THREADS / 32);
    if (precision_bytes == 4)
        k_reduce<float><<<rb + cb, RB_THREADS, 0, st>>>(O, nxpart, nzpart, nx, nz, zbc, rb, row_sum, col_sum, ticket,
                                                        out, avg, accumulate, 1.0 / nx, 1.0 / nz);
    else
        k_reduce<double><<<rb + cb, RB_THREADS, 0, st>>>(O, nxpart, nzpart, nx, nz, zbc, rb, row_sum, col_sum, ticket,
                                                         out, avg, accumulate, 1.0 / nx, 1.0 / nz);
    return cudaGetLastError();
}

template cudaError_t launch_init<float>(int, float*, const double*, const double*, const StepConst<float>&, cudaStream_t);
template cudaError_t launch_init<double>(int, double*, const double*, const double*, const StepConst<double>&,
                                         cudaStream_t);
template cudaError_t launch_export<float>(int, const float*, double*, const StepConst<float>&, cudaStream_t);
template cudaError_t launch_export<double>(int, const double*, double*, const StepConst<double>&, cudaStream_t);

}  // namespace lbm
