// lbm_twopass.cu -- the time step as two kernels: a density/psi pass, then a collide-and-push
// pass that stages the psi/rho halo tile in shared memory with a TMA tensor load.
//
// K1 (k_density) reads each site's populations once and writes rho_s and psi_s into padded
// field planes with 2 ghost rows and GX ghost columns on each side, filled with the periodic
// images or (with walls) the mirror images of the fluid, so that every tile of K2 is one
// in-bounds rectangle.  K2 (k_twopass) loads the (TPX + 8) x (TPZ + 4) tile of all fields with
// one cp.async.bulk.tensor (completion on an mbarrier, waited on with a bounded spin), reads
// its own populations from HBM, and runs the same per-site arithmetic as the fused kernel.
// HBM traffic per site-update: 2 x 9 x NS populations plus the fields written and read once
// (compare 2 x 9 x NS for the fused sweep).
#include <cuda.h>
#include <cudaTypedefs.h>

#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// ---- K1 ------------------------------------------------------------------------------------

// Ghost positions fed by site (x, z): every padded row zg (z + 2 plus ghost rows whose source
// row is z) times every padded column xg (x + GX plus ghost columns whose source column is x).
template <typename T, int NS>
__global__ void __launch_bounds__(256) k_density(const T* __restrict__ f, T* __restrict__ g, const StepConst<T> C,
                                                 const GhostGeom GG) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int z = blockIdx.y;
    if (x >= C.nx) return;
    const int nx = C.nx, nz = C.nz;
    T rho[NS], psi[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        T v[9];
#pragma unroll
        for (int l = 0; l < 9; ++l) v[l] = f[(s * 9 + l) * C.plane + (long long)z * C.pitch + x];
        rho[s] = C.rho_ref[s] + sum9(v);
        psi[s] = psi_of(C, s, rho[s]);
    }
    int rows[5], nr = 0;
    rows[nr++] = z + 2;
    for (int zr = -2; zr <= nz + 1; zr = (zr == -1 ? nz : zr + 1)) {
        int src;
        if (C.zbc == 0)
            src = wrap_index(zr, nz);
        else
            src = C.psi_wall == 1 ? -1 : mirror_index(zr, nz);
        if (src == z && nr < 5) rows[nr++] = zr + 2;
    }
    int cols[2 * GX + 1], nc = 0;
    cols[nc++] = x + GX;
    if (x < GX || x >= nx - GX) {
        for (int xc = -GX; xc < nx + GX; xc = (xc == -1 ? (nx > GX ? nx : 0) : xc + 1)) {
            if (xc >= 0 && xc < nx) continue;
            if (wrap_index(xc, nx) == x && nc < 2 * GX + 1) cols[nc++] = xc + GX;
        }
    }
    for (int a = 0; a < nr; ++a)
        for (int b = 0; b < nc; ++b) {
            const long long o = (long long)rows[a] * GG.gpitch + cols[b];
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                g[s * GG.gplane + o] = psi[s];
                g[(NS + s) * GG.gplane + o] = rho[s];
            }
        }
}

// ---- K2 ------------------------------------------------------------------------------------

constexpr int TW = TPX + 2 * GX;  // tile width in the field planes
constexpr int TH = TPZ + 4;       // tile height

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

template <typename T, int NS, int MODE>
__global__ void __launch_bounds__(TPX* TPZ) k_twopass(const T* __restrict__ fin, T* __restrict__ fout,
                                                      const StepConst<T> C, const __grid_constant__ CUtensorMap tmap,
                                                      const ObsPtrs O, int nxpart, int nzpart) {
    constexpr int NQF = 2 * NS;
    __shared__ __align__(128) T tile[NQF][TH][TW];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ T colsum[TPZ][NQC][TPX];
    __shared__ int timed_out;
    const int tx = threadIdx.x, tz = threadIdx.y, tid = tz * TPX + tx;
    const int x0 = blockIdx.x * TPX, z0 = blockIdx.y * TPZ;
    const int x = x0 + tx, z = z0 + tz;
    const int nx = C.nx, nz = C.nz;
    const long long plane = C.plane;
    const unsigned bar_a = smem_u32(&bar);

    if (tid == 0) {
        timed_out = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        constexpr unsigned bytes = (unsigned)(sizeof(T) * NQF * TH * TW);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar_a), "r"(bytes) : "memory");
        // field coordinates of the tile: column x0 (= x0 - GX in lattice columns), row z0 (= z0 - 2)
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
            "[%5];\n" ::"r"(smem_u32(&tile[0][0][0])),
            "l"(&tmap), "r"(x0), "r"(z0), "r"(0), "r"(bar_a)
            : "memory");
    }
    // meanwhile: this site's populations from HBM
    const bool live = x < nx && z < nz;
    T f[NS][9];
    if (live) {
        const T* base = fin + (long long)z * C.pitch + x;
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int l = 0; l < 9; ++l) f[s][l] = __ldg(base + (s * 9 + l) * plane);
    }
    // bounded wait for the tile (about 1 s at 2 GHz); on expiry flag LBM_ETIMEOUT and skip
    {
        const long long t0 = clock64();
        unsigned done = 0;
        while (!done) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(bar_a)
                : "memory");
            if (!done && clock64() - t0 > 2000000000LL) {
                timed_out = 1;
                break;
            }
        }
    }
    __syncthreads();
    if (timed_out) {
        if (tid == 0) atomicOr(O.flag, 2);
        return;
    }

    T F[NS][2];
    T sxx = T(0), szz = T(0), sxz = T(0);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        T p[5][5];
#pragma unroll
        for (int dz = 0; dz < 5; ++dz)
#pragma unroll
            for (int dx = 0; dx < 5; ++dx) p[dz][dx] = tile[s][tz + dz][tx + GX - 2 + dx];
        intra_force(C, s, p, F[s][0], F[s][1]);
        if (MODE & M_OBS) intra_stress(C, s, p, sxx, szz, sxz);
    }
    if constexpr (NS == 2) {
        T ra[3][3], rb[3][3];
#pragma unroll
        for (int dz = 0; dz < 3; ++dz)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                ra[dz][dx] = tile[2][tz + 1 + dz][tx + GX - 1 + dx];
                rb[dz][dx] = tile[3][tz + 1 + dz][tx + GX - 1 + dx];
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
        T drho[NS], rho[NS], ir[NS], jx[NS], jz[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            drho[s] = sum9(f[s]);
            rho[s] = C.rho_ref[s] + drho[s];
            if (!(rho[s] > T(0)) || !(rho[s] < T(1e30))) bad = 1;
            ir[s] = div_(T(1), rho[s]);
            momentum9(f[s], jx[s], jz[s]);
            F[s][0] += rho[s] * C.g;
        }
        if (MODE & M_OBS) {
            T ux, uz, pixz, rtot, mx, mz;
            site_kinetics<T, NS>(C, f, rho, ir, jx, jz, F, ux, uz, pixz, rtot, mx, mz);
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
        collide<T, NS>(C, f, drho, rho, ir, jx, jz, F);
        const bool wall_row = C.zbc == 1 && (z == 0 || z == nz - 1);
        const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
        const long long rz0 = (long long)z * C.pitch;
        const long long rzm = (long long)(z == 0 ? nz - 1 : z - 1) * C.pitch;
        const long long rzp = (long long)(z == nz - 1 ? 0 : z + 1) * C.pitch;
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int l = 0; l < 9; ++l) {
                const int col = cx(l) < 0 ? xm : (cx(l) > 0 ? xp : x);
                const int zd = z + cz(l);
                if (wall_row && (zd < 0 || zd >= nz)) {
                    const int w = zd < 0 ? 0 : 1;
                    const T back = bounce<T>(l, f[s][l], rho[s], C.wall_u[w]);
                    fout[(s * 9 + opp(l)) * plane + rz0 + x] = back;
                    if (MODE & M_OBS) {
                        const T dm = T(cx(l)) * (f[s][l] + back);
                        if (w == 0)
                            rowq[QR_WALLB] += dm;
                        else
                            rowq[QR_WALLT] += dm;
                    }
                } else {
                    const long long row = cz(l) < 0 ? rzm : (cz(l) > 0 ? rzp : rz0);
                    fout[(s * 9 + l) * plane + row + col] = f[s][l];
                }
            }
    }
    if (__any_sync(FULL, bad) && tx == 0) atomicOr(O.flag, 1);
    if (MODE & M_OBS) {
        // per-row sums over the 32 sites of this warp (one tile row), fixed order
#pragma unroll
        for (int k = 0; k < NQR; ++k) {
            T v = rowq[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
            rowq[k] = v;
        }
        if (tx < NQR && z < nz) {
            T v = rowq[0];
#pragma unroll
            for (int k = 1; k < NQR; ++k)
                if (tx == k) v = rowq[k];
            static_cast<T*>(O.part_row)[((long long)z * nxpart + blockIdx.x) * NQR + tx] = v;
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

template <typename T, int NS, int MODE>
cudaError_t launch_tp(const T* fin, T* fout, const StepConst<T>& C, const CUtensorMap* tm, const ObsPtrs& O,
                      int nxpart, int nzpart, cudaStream_t st) {
    const dim3 block(TPX, TPZ), grid(nxpart, nzpart);
    k_twopass<T, NS, MODE><<<grid, block, 0, st>>>(fin, fout, C, *tm, O, nxpart, nzpart);
    return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_density(int ns, const T* f, T* g, const StepConst<T>& C, const GhostGeom& GG, cudaStream_t st) {
    const dim3 block(256), grid((C.nx + 255) / 256, C.nz);
    if (ns == 1)
        k_density<T, 1><<<grid, block, 0, st>>>(f, g, C, GG);
    else
        k_density<T, 2><<<grid, block, 0, st>>>(f, g, C, GG);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_twopass(int ns, int mode, const T* fin, T* fout, const T* /*gfield*/, const StepConst<T>& C,
                           const GhostGeom& /*GG*/, const void* tmap, const ObsPtrs& O, int nxpart, int nzpart,
                           cudaStream_t st) {
    const CUtensorMap* tm = static_cast<const CUtensorMap*>(tmap);
    if (ns == 1) {
        if (mode == M_WRITE) return launch_tp<T, 1, M_WRITE>(fin, fout, C, tm, O, nxpart, nzpart, st);
        if (mode == (M_WRITE | M_OBS)) return launch_tp<T, 1, M_WRITE | M_OBS>(fin, fout, C, tm, O, nxpart, nzpart, st);
    } else {
        if (mode == M_WRITE) return launch_tp<T, 2, M_WRITE>(fin, fout, C, tm, O, nxpart, nzpart, st);
        if (mode == (M_WRITE | M_OBS)) return launch_tp<T, 2, M_WRITE | M_OBS>(fin, fout, C, tm, O, nxpart, nzpart, st);
    }
    return cudaErrorInvalidValue;
}

// Tensor map of the field planes [2 ns][nz + 4][gpitch], box (TPX + 2 GX) x (TPZ + 4) x 2 ns.
void* tensor_map_encoder() {
    static void* encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return nullptr;
        encode = fn;
    }
    return encode;
}

int make_field_tmap(void* out, const void* g, int esize, int ns, int nz, const GhostGeom& GG) {
    const auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encoder());
    if (!encode) return 1;
    const cuuint64_t dims[3] = {(cuuint64_t)GG.gpitch, (cuuint64_t)(nz + 4), (cuuint64_t)(2 * ns)};
    const cuuint64_t strides[2] = {(cuuint64_t)GG.gpitch * esize, (cuuint64_t)GG.gplane * esize};
    const cuuint32_t box[3] = {(cuuint32_t)TW, (cuuint32_t)TH, (cuuint32_t)(2 * ns)};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode(static_cast<CUtensorMap*>(out),
                              esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                              const_cast<void*>(g), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : 2;
}

template cudaError_t launch_density<float>(int, const float*, float*, const StepConst<float>&, const GhostGeom&,
                                           cudaStream_t);
template cudaError_t launch_density<double>(int, const double*, double*, const StepConst<double>&, const GhostGeom&,
                                            cudaStream_t);
template cudaError_t launch_twopass<float>(int, int, const float*, float*, const float*, const StepConst<float>&,
                                           const GhostGeom&, const void*, const ObsPtrs&, int, int, cudaStream_t);
template cudaError_t launch_twopass<double>(int, int, const double*, double*, const double*, const StepConst<double>&,
                                            const GhostGeom&, const void*, const ObsPtrs&, int, int, cudaStream_t);

}  // namespace lbm
