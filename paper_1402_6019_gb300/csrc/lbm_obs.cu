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

// One warp per row: the row's totals over its column groups, its profile entries
// (x-averages), its fluidity (Eq. fluidity: shear rate = central difference of ux_z, one-sided
// at wall rows, wrapped when periodic, over the shear stress) and, when sampling, its time
// sums.  One warp per column: the z-averages of P_xx - P_zz and P_xx.  Each block folds the
// scalar contributions of its rows (mass A, B, momentum x, z) or columns (gamma) into one
// FP64 partial; the last block to finish sums the block partials.  Group sums within a row or
// a column stay in the populations' precision PT (in FP32 mode they are sums of FP32 values;
// FP64 arithmetic is scarce on this GPU, so the FP64 work is spread over all blocks); each
// total is widened to FP64 once.  Every sum runs in a fixed order: repeatable results.
template <typename PT>
__global__ void __launch_bounds__(RB_THREADS) k_reduce(const ObsPtrs O, int nxpart, int nzpart, int nx, int nz, int zbc,
                                                       int nrowblocks, double* __restrict__ walls,
                                                       double* __restrict__ bpart, unsigned* ticket,
                                                       double* __restrict__ out, double* __restrict__ avg,
                                                       int accumulate, double inx, double inz) {
    constexpr int WPB = RB_THREADS / 32;
    __shared__ double wsc[WPB][NSC];
    __shared__ double fin[NSC][RB_THREADS];
    __shared__ bool last;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const PT* const prow = static_cast<const PT*>(O.part_row);
    const PT* const pcol = static_cast<const PT*>(O.part_col);
    double* const ux = out + O_PROF;
    double* const rz = ux + nz;
    double* const sx = rz + 2LL * nz;
    double* const fl = sx + nz;
    double* const ps = fl + nz;
    double* const px = ps + nx;
    for (int k = lane; k < NSC; k += 32) wsc[warp][k] = 0.0;
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
            // lanes 0..8 finish one output each
            if (lane <= NQR) {
                PT mine = v[0];
#pragma unroll
                for (int k = 1; k < NQR; ++k)
                    if (lane == k) mine = v[k];
                const double d = (double)mine;
                switch (lane) {
                    case QR_UX:
                        ux[z] = d * inx;
                        if (accumulate) avg[O_PROF + z] += d * inx;
                        break;
                    case QR_RHOA:
                        rz[z] = d * inx;
                        wsc[warp][0] = d;
                        if (accumulate) avg[O_PROF + nz + z] += d * inx;
                        break;
                    case QR_RHOB:
                        rz[nz + z] = d * inx;
                        wsc[warp][1] = d;
                        if (accumulate) avg[O_PROF + 2LL * nz + z] += d * inx;
                        break;
                    case QR_SXZ:
                        sx[z] = d * inx;
                        if (accumulate) avg[O_PROF + 3LL * nz + z] += d * inx;
                        break;
                    case QR_MX: wsc[warp][2] = d; break;
                    case QR_MZ: wsc[warp][3] = d; break;
                    case QR_WALLB: if (z == 0) walls[0] = d; break;
                    case QR_WALLT: if (z == nz - 1) walls[1] = d; break;
                    case NQR: {  // fluidity
                        const double gd =
                            nz == 1 ? 0.0 : (wr * (double)v[NQR + 1] - wl * (double)v[NQR]) * inx;
                        const double f = gd / ((double)v[QR_SXZ] * inx);
                        fl[z] = f;
                        if (accumulate) avg[O_PROF + 4LL * nz + z] += f;
                        break;
                    }
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
                const double a = (double)v[QC_PS] * inz;
                ps[x] = a;
                wsc[warp][4] = a;
                if (accumulate) avg[O_PROF + 5LL * nz + x] += a;
            } else if (lane == 1) {
                const double b = (double)v[QC_PXX] * inz;
                px[x] = b;
                if (accumulate) avg[O_PROF + 5LL * nz + nx + x] += b;
            }
        }
    }
    __syncthreads();
    if (t < NSC) {  // this block's share of the scalars, warps in order
        double a = 0.0;
        for (int w = 0; w < WPB; ++w) a += wsc[w][t];
        bpart[(long long)blockIdx.x * NSC + t] = a;
    }
    // the block's writes happen before thread 0's fence (barrier); the fence is cumulative, so
    // the block drawing the last ticket sees every block's results
    __syncthreads();
    if (t == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
        if (last) __threadfence();
    }
    __syncthreads();
    if (!last) return;
    double acc[NSC] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = t; b < (int)gridDim.x; b += RB_THREADS)
        for (int k = 0; k < NSC; ++k) acc[k] += bpart[(long long)b * NSC + k];
    for (int k = 0; k < NSC; ++k) fin[k][t] = acc[k];
    __syncthreads();
    for (int o = RB_THREADS / 2; o > 0; o >>= 1) {
        if (t < o)
            for (int k = 0; k < NSC; ++k) fin[k][t] += fin[k][t + o];
        __syncthreads();
    }
    if (t == 0) {
        const double m0 = fin[0][0], m1 = fin[1][0], mx = fin[2][0], mz = fin[3][0], g = fin[4][0];
        out[O_MASS] = m0;
        out[O_MASS + 1] = m1;
        out[O_MOM] = mx;
        out[O_MOM + 1] = mz;
        out[O_GAMMA] = g;
        out[O_WALL] = zbc ? walls[0] * inx : 0.0;
        out[O_WALL + 1] = zbc ? walls[1] * inx : 0.0;
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
                          double* walls, double* bpart, unsigned* ticket, double* out, double* avg, int accumulate,
                          cudaStream_t st) {
    const int rb = (nz + RB_THREADS / 32 - 1) / (RB_THREADS / 32);
    const int cb = (nx + RB_THREADS / 32 - 1) / (RB_THREADS / 32);
    const double inx = 1.0 / nx, inz = 1.0 / nz;
    if (precision_bytes == 4)
        k_reduce<float><<<rb + cb, RB_THREADS, 0, st>>>(O, nxpart, nzpart, nx, nz, zbc, rb, walls, bpart, ticket, out,
                                                        avg, accumulate, inx, inz);
    else
        k_reduce<double><<<rb + cb, RB_THREADS, 0, st>>>(O, nxpart, nzpart, nx, nz, zbc, rb, walls, bpart, ticket, out,
                                                         avg, accumulate, inx, inz);
    return cudaGetLastError();
}

template cudaError_t launch_init<float>(int, float*, const double*, const double*, const StepConst<float>&, cudaStream_t);
template cudaError_t launch_init<double>(int, double*, const double*, const double*, const StepConst<double>&,
                                         cudaStream_t);
template cudaError_t launch_export<float>(int, const float*, double*, const StepConst<float>&, cudaStream_t);
template cudaError_t launch_export<double>(int, const double*, double*, const StepConst<double>&, cudaStream_t);

}  // namespace lbm
