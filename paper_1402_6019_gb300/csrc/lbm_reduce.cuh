// lbm_reduce.cuh -- the FP64-grade reduction of the step kernels' partial sums into the
// observables, as a block-level routine: run by the reduction kernel (one block per work item)
// and, folded into the next time step, by the pull kernel's CTAs.
#pragma once

#include "lbm_internal.h"

namespace lbm {

constexpr int RB_THREADS = 256;
constexpr int NSC = 5;  // scalar slots per row / column: mass A, mass B, momentum x, z; gamma

template <typename PT>
__device__ PT warp_sum(PT v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Accumulators of the reduction.  FP64 mode: plain doubles.  FP32 mode: double-float pairs
// (hi + lo, compensated summation with Knuth's TwoSum on the FP32 pipes, about 48 significant
// bits) -- the FP64 unit of this GPU has long latency and low throughput, and on the
// reduction's short dependent chains each FP64 operation cost microseconds, so in FP32 mode no
// FP64 arithmetic is issued; the host widens hi + lo to FP64.  Entry i of `out` and `avg` is an
// 8-byte double (FP64 mode) or an 8-byte (hi, lo) float pair (FP32 mode).
__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, e);
}
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
    const float2 s = two_sum(a.x, b.x);
    const float lo = __fadd_rn(s.y, __fadd_rn(a.y, b.y));
    const float hi = __fadd_rn(s.x, lo);
    return make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, s.x)));
}

template <typename PT> struct Red;
template <> struct Red<double> {
    using A = double;
    __device__ static A zero() { return 0.0; }
    __device__ static A from(double v) { return v; }
    __device__ static A add(A a, A b) { return a + b; }
    __device__ static void put(void* buf, long long i, A v) { static_cast<double*>(buf)[i] = v; }
    __device__ static void acc(void* buf, long long i, A v) { static_cast<double*>(buf)[i] += v; }
    __device__ static A get(const void* buf, long long i) { return static_cast<const double*>(buf)[i]; }
    __device__ static bool finite(A a) { return isfinite(a); }
    __device__ static bool nonzero(A a) { return a != 0.0; }
};
template <> struct Red<float> {
    using A = float2;
    __device__ static A zero() { return make_float2(0.f, 0.f); }
    __device__ static A from(float v) { return make_float2(v, 0.f); }
    __device__ static A add(A a, A b) { return ff_add(a, b); }
    __device__ static void put(void* buf, long long i, A v) { static_cast<float2*>(buf)[i] = v; }
    __device__ static void acc(void* buf, long long i, A v) {
        float2* p = static_cast<float2*>(buf) + i;
        *p = ff_add(*p, v);
    }
    __device__ static A get(const void* buf, long long i) { return static_cast<const float2*>(buf)[i]; }
    __device__ static bool finite(A a) { return isfinite(a.x) && isfinite(a.y); }
    __device__ static bool nonzero(A a) { return a.x != 0.f || a.y != 0.f; }
};

// Work item blk, run by a block of RB_THREADS threads (all of which call this), or with WIDE by a
// block of a multiple of them, whose warps past the first RB_THREADS / 32 take part in the
// barriers only.  One warp per
// row: the row's totals over its column groups, its profile entries (x-averages), its fluidity (Eq. fluidity: shear rate = central difference of ux_z, one-sided
// at wall rows, wrapped when periodic, over the shear stress), its wall momenta and, when
// sampling, its time sums.  One warp per column: the z-averages of P_xx - P_zz and P_xx.  Each
// block folds the scalar contributions of its rows (mass A, B, momentum x, z) or columns
// (gamma) into one partial, stored after the profiles (and added to its own time sum).  The
// sum over blocks is left to the reader (the host sums the block partials in FP64), except
// with TAIL, where the last block to finish writes the scalars into `out` on the device.
// accumulate: 0 = `out` and `bpart` only; 1 = also add the sample to the time sums `avg` and
// `bavg`; 2 = also write the sample into `avg` and `bavg` in place of what they held (a record
// of this one sample, with its bad-density flag).
// Group sums within a row or a column stay in the populations' precision PT; time sums and
// block partials use the accumulators above.  Fixed summation order: repeatable results.
// inst / ninst: the lattices of a stacked batch (rows of different lattices are not neighbours);
// null for a single lattice of nz rows.
template <typename PT, bool WIDE = false>
__device__ __forceinline__ void reduce_block(int blk, const void* part_row, const void* part_col, const int* flag,
                                             int nxpart, int nzpart, int nx, int nz, int zbc, int nrowblocks,
                                             void* __restrict__ out, void* __restrict__ avg,
                                             void* __restrict__ bpart, void* __restrict__ bavg, int accumulate,
                                             PT inx, PT inz, typename Red<PT>::A (*wsc)[NSC],
                                             const InstGeom* __restrict__ inst = nullptr, int ninst = 0) {
    using R = Red<PT>;
    using A = typename R::A;
    constexpr int WPB = RB_THREADS / 32;
    const int t = (int)(threadIdx.y * blockDim.x + threadIdx.x), lane = t & 31, warp = t >> 5;
    const PT* const prow = static_cast<const PT*>(part_row);
    const PT* const pcol = static_cast<const PT*>(part_col);
    const long long iux = O_PROF, irz = O_PROF + nz, isx = O_PROF + 3LL * nz, ifl = O_PROF + 4LL * nz,
                    ips = O_PROF + 5LL * nz, ipx = ips + nx, imx = ipx + nx, imz = imx + nz, iwb = imz + nz,
                    iwt = iwb + nz;
    for (int k = lane; k < NSC; k += 32) wsc[warp][k] = R::zero();
    if (blk == 0 && t == 0) {  // the step kernels' flag of a bad density
        const bool bad = (flag[0] & 1) != 0;
        R::put(out, O_BAD, R::from(bad ? PT(1) : PT(0)));
        if (accumulate == 2)
            R::put(avg, O_BAD, R::from(bad ? PT(1) : PT(0)));
        else if (accumulate && bad)
            R::put(avg, O_BAD, R::from(PT(1)));
    }
    if (WIDE && warp >= WPB) {
        // idle in this work item
    } else if (blk < nrowblocks) {
        const int z = blk * WPB + warp;
        if (z < nz) {
            // this row's lattice: its first compact row and height
            int z0 = 0, nzi = nz;
            if (inst) {
                const int k = inst_of_row(inst, ninst, z);
                z0 = inst[k].zrow0;
                nzi = inst[k].nz;
            }
            const int zi = z - z0;  // row within the lattice
            int zl = zi - 1, zr = zi + 1;
            PT wl = PT(0.5), wr = PT(0.5);
            if (nzi == 1) {
                zl = zr = zi;
            } else if (zbc == 0) {
                zl = zi == 0 ? nzi - 1 : zi - 1;
                zr = zi == nzi - 1 ? 0 : zi + 1;
            } else if (zi == 0) {
                zl = 0;
                wl = wr = PT(1);
            } else if (zi == nzi - 1) {
                zr = nzi - 1;
                wl = wr = PT(1);
            }
            zl += z0;
            zr += z0;
            // the output entries of this lane (lanes 0..8), -1 for none; the second is the wall
            // force scalar of a single lattice
            long long oi = -1, oi2 = -1;
            switch (lane) {
                case QR_UX: oi = iux + z; break;
                case QR_RHOA: oi = irz + z; break;
                case QR_RHOB: oi = irz + nz + z; break;
                case QR_SXZ: oi = isx + z; break;
                case QR_MX: oi = imx + z; break;
                case QR_MZ: oi = imz + z; break;
                case QR_WALLB:
                    oi = iwb + z;
                    oi2 = (!inst && zbc && z == 0) ? O_WALL : -1;
                    break;
                case QR_WALLT:
                    oi = iwt + z;
                    oi2 = (!inst && zbc && z == nz - 1) ? O_WALL + 1 : -1;
                    break;
                case NQR: oi = ifl + z; break;
                default: break;
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
            const A old = (accumulate == 1 && oi >= 0) ? R::get(avg, oi) : R::zero();  // in flight with the sums
            const A old2 = (accumulate == 1 && oi2 >= 0) ? R::get(avg, oi2) : R::zero();
#pragma unroll
            for (int k = 0; k < NQR + 2; ++k) v[k] = warp_sum(v[k]);
            if (lane <= NQR) {
                PT mine = v[0];
#pragma unroll
                for (int k = 1; k < NQR; ++k)
                    if (lane == k) mine = v[k];
                A val;
                if (lane == NQR) {  // fluidity
                    const PT gd = nzi == 1 ? PT(0) : (wr * v[NQR + 1] - wl * v[NQR]) * inx;
                    val = R::from(gd / (v[QR_SXZ] * inx));
                } else {
                    val = R::from(mine * inx);
                }
                if (lane == QR_RHOA) wsc[warp][0] = R::from(mine);
                if (lane == QR_RHOB) wsc[warp][1] = R::from(mine);
                if (lane == QR_MX) wsc[warp][2] = R::from(mine);
                if (lane == QR_MZ) wsc[warp][3] = R::from(mine);
                if (oi >= 0) {
                    R::put(out, oi, val);
                    if (accumulate) R::put(avg, oi, R::add(old, val));
                }
                if (oi2 >= 0) {
                    R::put(out, oi2, val);
                    if (accumulate) R::put(avg, oi2, R::add(old2, val));
                }
            }
        }
    } else {
        const int x = (blk - nrowblocks) * WPB + warp;
        if (x < nx) {
            const long long oi = lane == 0 ? ips + x : (lane == 1 ? ipx + x : -1);
            PT v[NQC];
#pragma unroll
            for (int k = 0; k < NQC; ++k) v[k] = PT(0);
            for (int p = lane; p < nzpart; p += 32) {
                const PT* src = pcol + ((long long)x * nzpart + p) * NQC;
#pragma unroll
                for (int k = 0; k < NQC; ++k) v[k] += src[k];
            }
            const A old = (accumulate == 1 && oi >= 0) ? R::get(avg, oi) : R::zero();
#pragma unroll
            for (int k = 0; k < NQC; ++k) v[k] = warp_sum(v[k]);
            if (oi >= 0) {
                const A val = R::from((lane == 0 ? v[QC_PS] : v[QC_PXX]) * inz);
                if (lane == 0) wsc[warp][4] = val;
                R::put(out, oi, val);
                if (accumulate) R::put(avg, oi, R::add(old, val));
            }
        }
    }
    __syncthreads();
    A bsum = R::zero();
    if (t < NSC) {  // this block's share of the scalars, warps in order
        const long long i = (long long)blk * NSC + t;
        const A old = accumulate == 1 ? R::get(bavg, i) : R::zero();
        for (int w = 0; w < WPB; ++w) bsum = R::add(bsum, wsc[w][t]);
        R::put(bpart, i, bsum);
        if (accumulate) R::put(bavg, i, R::add(old, bsum));
    }
    __syncthreads();  // wsc may be reused by the caller's next work item
}

}  // namespace lbm
