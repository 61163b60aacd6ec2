// lbm_fused.cu -- one-pass time step of the multirange Shan-Chen lattice Boltzmann model.
//
// One warp owns a strip of STRIP_W = 28 columns plus a 2-column halo on each side (the reach
// of the 5x5 stencil of Eq. FORCE) and sweeps a chunk of rows in z.  Each lane copies the
// 9 (x species) populations of its column for row r + PF + 1 into a per-warp ring in shared
// memory with cp.async while it works on row r (PF rows in flight beyond the current one), so
// HBM reads are coalesced (x fastest) and overlapped with compute.  From the ring it forms
// the density and psi of row r and keeps psi and rho of the last five rows in registers.  Two
// rows behind, the row is complete: the lanes gather the 5x5 psi and 3x3 rho neighbourhoods
// with warp shuffles, form the force (Eq. FORCE + cross term + body force), and the 28 owned
// lanes read their populations back from the ring, collide (Eq. LB with the shifted velocity
// of Sec. II) and push them to their neighbours (streaming, with the halfway bounce-back
// walls of Sec. IV).  Compared with a psi pass followed by a collide pass this moves each
// population once in and once out of HBM per step.  A lane only ever reads ring entries it
// copied itself.
//
// With M_OBS the same pass also accumulates the observables of the state being collided:
// per-row sums over the strip (warp reduction) and per-column sums over the chunk.
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// rows in flight beyond the current one, and ring depth (current row, the two rows behind it
// that are still to be collided, the row being overwritten, and the prefetched rows)
template <typename T> constexpr int prefetch_rows() { return sizeof(T) == 4 ? 2 : 1; }
template <typename T> constexpr int ring_rows() { return prefetch_rows<T>() + 4; }
constexpr int WARPS_PER_BLOCK = 4;

template <typename T, int NS>
constexpr int ring_bytes_per_block() {
    return WARPS_PER_BLOCK * ring_rows<T>() * NS * 9 * 32 * (int)sizeof(T);
}

template <typename T>
__device__ __forceinline__ void cp_async(T* smem, const T* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename T, int NS, int MODE>
__global__ void __launch_bounds__(128) k_fused(const T* __restrict__ fin, T* __restrict__ fout,
                                               const StepConst<T> C, const SweepGeom G, const ObsPtrs O) {
    constexpr int PF = prefetch_rows<T>();
    constexpr int RS = ring_rows<T>();
    constexpr int ROWV = NS * 9 * 32;  // ring values per row: [species*9 + l][lane]
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* const ring = reinterpret_cast<T*>(smem_raw) + (threadIdx.x >> 5) * RS * ROWV;
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

    // ring slots (rolling): row r lives in slot (r - (z0 - 2)) mod RS
    T* const lane_ring = ring + lane;
    int s_issue = 0;  // slot of the next row to issue
    int s_cur = 0;    // slot of the current row r
    int s_col = RS - 2 < 0 ? 0 : RS - 2;  // slot of row r - 2 (meaningful once r - 2 >= z0)
    // asynchronous copy of this lane's column of row r into the ring (one commit group per row)
    auto issue = [&](int r) {
        if (r <= z1 + 1) {
            const int rr = source_row(C, r);
            if (rr >= 0) {
                T* dst = lane_ring + s_issue * ROWV;
                const T* src = fin + (long long)rr * pitch + xw;
#pragma unroll
                for (int k = 0; k < NS * 9; ++k) cp_async(dst + k * 32, src + k * plane);
            }
        }
        cp_async_commit();
        s_issue = s_issue + 1 == RS ? 0 : s_issue + 1;
    };
#pragma unroll
    for (int i = 0; i <= PF; ++i) issue(z0 - 2 + i);

    for (int r = z0 - 2; r <= z1 + 1; ++r) {
        issue(r + PF + 1);
        cp_async_wait<PF + 1>();  // row r has landed
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
                const T* base = lane_ring + s_cur * ROWV;
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    T f[9];
#pragma unroll
                    for (int l = 0; l < 9; ++l) f[l] = base[(s * 9 + l) * 32];
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
        const int s_z = s_col;  // slot of row z
        s_col = s_col + 1 == RS ? 0 : s_col + 1;
        s_cur = s_cur + 1 == RS ? 0 : s_cur + 1;
        if (z < z0) {  // prologue rows (warp-uniform)
            __syncwarp();
            continue;
        }

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
            T f[NS][9], drho[NS], rho[NS], ir[NS], jx[NS], jz[NS];
            const T* base = lane_ring + s_z * ROWV;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
#pragma unroll
                for (int l = 0; l < 9; ++l) f[s][l] = base[(s * 9 + l) * 32];
                drho[s] = dr[s][2];
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
                const bool wall_row = C.zbc == 1 && (z == 0 || z == nz - 1);  // warp-uniform
                if ((MODE & M_WRITE) || wall_row) {
                    collide<T, NS>(C, f, drho, rho, ir, jx, jz, F);
                    // streaming: f_l(x + c_l) = g_l(x), periodic in x, periodic or walls in z
                    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
                    const long long rz0 = (long long)z * pitch;
                    const long long rzm = (long long)(z == 0 ? nz - 1 : z - 1) * pitch;
                    const long long rzp = (long long)(z == nz - 1 ? 0 : z + 1) * pitch;
                    if (!wall_row) {
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
                                    if (MODE & M_OBS) {  // constant indices keep rowq in registers
                                        const T dm = T(cx(l)) * (f[s][l] + back);
                                        if (w == 0)
                                            rowq[QR_WALLB] += dm;
                                        else
                                            rowq[QR_WALLT] += dm;
                                    }
                                } else if (MODE & M_WRITE) {
                                    fout[(s * 9 + l) * plane + (long long)zd * pitch + col] = f[s][l];
                                }
                            }
                    }
                }
            }
        }
        if (MODE & M_OBS) {
            // transpose-reduce of the NQR = 8 row quantities over the 32 lanes: each halving
            // step exchanges half of the remaining values, 4 + 2 + 1 + 1 + 1 shuffles in all;
            // afterwards lane 4q holds the warp sum of quantity q (fixed order: repeatable)
            static_assert(NQR == 8, "row reduction is written for 8 quantities");
            T v4[4], v2[2], v1;
            const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
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
            if ((lane & 3) == 0) {
                const int q = (b4 ? 4 : 0) + (b3 ? 2 : 0) + (b2 ? 1 : 0);
                static_cast<T*>(O.part_row)[((long long)z * G.nstrips + strip) * NQR + q] = v1;
            }
        }
        __syncwarp();  // ring slots read this iteration may be refilled by the next issue
    }
    cp_async_wait<0>();
    if ((MODE & M_OBS) && owned) {
        T* dst = static_cast<T*>(O.part_col) + ((long long)x * G.nchunks + chunk) * NQC;
        dst[QC_PS] = acc_ps;
        dst[QC_PXX] = acc_pxx;
    }
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(O.flag, 1);
}

template <typename T, int NS, int MODE>
cudaError_t launch_mode(const T* fin, T* fout, const StepConst<T>& C, const SweepGeom& G, const ObsPtrs& O,
                        cudaStream_t st) {
    constexpr int smem = ring_bytes_per_block<T, NS>();
    static bool configured = false;  // per instantiation; the attribute is per function
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_fused<T, NS, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int warps = G.nstrips * G.nchunks;
    const dim3 block(32 * WARPS_PER_BLOCK), grid((warps + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK);
    k_fused<T, NS, MODE><<<grid, block, smem, st>>>(fin, fout, C, G, O);
    return cudaGetLastError();
}

template <typename T, int NS, int MODE>
int resident_mode(int nsm) {
    constexpr int smem = ring_bytes_per_block<T, NS>();
    if (cudaFuncSetAttribute(k_fused<T, NS, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_fused<T, NS, MODE>, 32 * WARPS_PER_BLOCK, smem) !=
        cudaSuccess)
        return 0;
    return blocks * WARPS_PER_BLOCK * nsm;
}

template <typename T, int NS>
cudaError_t launch_ns(int mode, const T* fin, T* fout, const StepConst<T>& C, const SweepGeom& G, const ObsPtrs& O,
                      cudaStream_t st) {
    switch (mode) {
        case M_WRITE: return launch_mode<T, NS, M_WRITE>(fin, fout, C, G, O, st);
        case M_WRITE | M_OBS: return launch_mode<T, NS, M_WRITE | M_OBS>(fin, fout, C, G, O, st);
        case M_OBS: return launch_mode<T, NS, M_OBS>(fin, fout, C, G, O, st);
        case M_FIELDS: return launch_mode<T, NS, M_FIELDS>(fin, fout, C, G, O, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_fused(int ns, int mode, const T* fin, T* fout, const StepConst<T>& C, const SweepGeom& G,
                         const ObsPtrs& O, cudaStream_t st) {
    return ns == 1 ? launch_ns<T, 1>(mode, fin, fout, C, G, O, st) : launch_ns<T, 2>(mode, fin, fout, C, G, O, st);
}

template <typename T>
int fused_resident_warps(int ns, int mode, int nsm) {
    if (ns == 1)
        return mode & M_OBS ? resident_mode<T, 1, M_WRITE | M_OBS>(nsm) : resident_mode<T, 1, M_WRITE>(nsm);
    return mode & M_OBS ? resident_mode<T, 2, M_WRITE | M_OBS>(nsm) : resident_mode<T, 2, M_WRITE>(nsm);
}

template int fused_resident_warps<float>(int, int, int);
template int fused_resident_warps<double>(int, int, int);

template cudaError_t launch_fused<float>(int, int, const float*, float*, const StepConst<float>&, const SweepGeom&,
                                         const ObsPtrs&, cudaStream_t);
template cudaError_t launch_fused<double>(int, int, const double*, double*, const StepConst<double>&,
                                          const SweepGeom&, const ObsPtrs&, cudaStream_t);

}  // namespace lbm
