// lbm3d.cu -- the three-dimensional extension of the two-belt Shan-Chen step (D3Q19; Eq. FORCE
// over the 3-D links of |c|^2 <= 8 with Appendix B's weights solved in three dimensions; the
// cross repulsion of Sec. IV over the first belt; the shifted-velocity BGK collision of
// Sec. II), behind the lbm3_* C ABI of include/lbm3d.h.
//
// A step is two kernels.
//  * k3_density reads each site's populations once and writes psi_s and rho_s into two
//    ghost-padded volumes (4 ghost columns in x, 2 ghost rows in y and z, holding the periodic
//    images, or beyond a wall the mirror images of the fluid), the two species of a site side
//    by side, so that a tile with its 2-cell halo is one in-bounds box.
//  * k3_step: a CTA of 32 x 4 x 2 sites loads the box of both volumes around its tile
//    (40 x 8 x 6 positions, x from x0 - 4 for 16-byte alignment) with one 4-D
//    cp.async.bulk.tensor on an mbarrier while every thread loads its own 19 populations per
//    species from HBM; then the force (46 antipodal link pairs, gathered shell by shell, both
//    species at once), the cross force, the collision, and the push of the new populations to
//    x + c_l (periodic in x and y, periodic or halfway bounce-back with Ladd's term in z).
// HBM traffic per site-update (FP32, two species): 152 B of populations read twice and written
// once plus the 16 B of the volumes written and read, 488 B; the method's own is 304 B
// (each population read and written once).  Populations are SoA f[s][l][z][y][x] (rows padded
// to 32), FP32 deviations f - W_l rho_ref,s or plain FP64.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm3d.h"
#include "lbm_internal.h"

namespace lbm3 {

// ---- lattice -------------------------------------------------------------------------------

// D3Q19: rest, +-x, +-y, +-z, then the 12 edges; every velocity is followed by its opposite.
// Each velocity is coded as (cx + 1) + 3 (cy + 1) + 9 (cz + 1).
__host__ __device__ constexpr int code19(int l) {
    constexpr int k[19] = {13, 14, 12, 16, 10, 22, 4, 17, 9, 11, 15, 23, 3, 5, 21, 25, 1, 7, 19};
    return k[l];
}
__host__ __device__ constexpr int c3x(int l) { return code19(l) % 3 - 1; }
__host__ __device__ constexpr int c3y(int l) { return code19(l) / 3 % 3 - 1; }
__host__ __device__ constexpr int c3z(int l) { return code19(l) / 9 - 1; }
__host__ __device__ constexpr int opp19(int l) { return l == 0 ? 0 : (l % 2 ? l + 1 : l - 1); }
// The first velocity with a nonzero component along an axis (0: x, 1: y, 2: z).
__host__ __device__ constexpr int first19(int axis) {
    for (int l = 1; l < 19; ++l)
        if ((axis == 0 ? c3x(l) : (axis == 1 ? c3y(l) : c3z(l))) != 0) return l;
    return 0;
}
// Every odd velocity's first nonzero component is +1, so c_l . u can start from that component.
__host__ __device__ constexpr bool odd_velocities_lead_positive() {
    for (int l = 1; l < 19; l += 2)
        if ((c3x(l) ? c3x(l) : (c3y(l) ? c3y(l) : c3z(l))) != 1) return false;
    return true;
}
static_assert(odd_velocities_lead_positive(), "c_l . u of an odd velocity starts from a +1 component");
static_assert(c3x(first19(0)) == 1 && c3y(first19(1)) == 1 && c3z(first19(2)) == 1,
              "the momentum sums start from a +1 component");
template <typename T>
__host__ __device__ constexpr T w19(int l) {
    return l == 0 ? T(1) / T(3) : (l <= 6 ? T(1) / T(18) : T(1) / T(36));
}

// Interaction weights by shell |c|^2 (Appendix B's constraints solved in three dimensions).
inline double w_att3(int q) {
    switch (q) {
        case 1: return 2.0 / 15.0;
        case 2: return 1.0 / 15.0;
        case 3: return 1.0 / 60.0;
        case 4: return 1.0 / 120.0;
        default: return 0.0;
    }
}
inline double w_rep3(int q) {
    switch (q) {
        case 1: return 4.0 / 45.0;
        case 2: return 1.0 / 21.0;
        case 3: return 2.0 / 105.0;
        case 4: return 5.0 / 504.0;
        case 5: return 1.0 / 315.0;
        case 6: return 1.0 / 630.0;
        case 8: return 1.0 / 5040.0;
        default: return 0.0;
    }
}
inline double w_cross3(int q) { return q == 1 ? 1.0 / 6.0 : (q == 2 ? 1.0 / 12.0 : 0.0); }

// ---- pairs of the two species ----------------------------------------------------------------

// A site's two species side by side: float2 (FP32, packed instructions) or double2.
template <typename T> struct PairOf;
template <> struct PairOf<float> { using V = float2; };
template <> struct PairOf<double> { using V = double2; };

__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vsplat(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 vswap(float2 a) { return make_float2(a.y, a.x); }
__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 vsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 vmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 vfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 vsplat(double a) { return make_double2(a, a); }
__device__ __forceinline__ double2 vswap(double2 a) { return make_double2(a.y, a.x); }

// Scalar operations whose rounding is fixed (the compiler neither contracts nor reorders them).
__device__ __forceinline__ float smul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double smul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float sadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double sadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double sfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// ---- geometry and constants ----------------------------------------------------------------

constexpr int GX = 4, GY = 2, GZ = 2;         // ghosts of the psi / rho volumes
constexpr int TX = 32;                        // tile width: one warp per tile row
constexpr int BX = TX + 2 * GX;               // box width (x from x0 - 4: 16-byte aligned)
constexpr long long WAIT_LIMIT = 2000000000LL;  // clock cycles of the bounded wait (~1 s)
// The tile shapes (TY x TZ rows of 32 sites, one thread per site) lbm3_autotune chooses from:
// the halo box of a tile is (TY + 4) x (TZ + 4) rows, so flatter tiles read more halo from L2
// per site and taller ones hold fewer CTAs per SM.
constexpr int NSHAPE = 4;
constexpr int SHAPE_TY[NSHAPE] = {4, 2, 8, 4};
constexpr int SHAPE_TZ[NSHAPE] = {2, 4, 1, 4};

template <typename T>
struct Step3 {
    int nx, ny, nz, ns, zbc, psi_form;
    int pitch;            // population row length (nx rounded up to 32)
    int gpitch;           // sites per row of a volume (nx + 2 GX rounded up to 4)
    long long plane;      // elements of one population volume (nz * ny * pitch)
    long long gvol;       // pairs in one psi / rho volume (gz * gy * gpitch)
    int gy, gz;           // rows and layers of a volume (ny + 2 GY, nz + 2 GZ)
    T omega[2], tau[2], rho_ref[2], inv_rho0[2], rho0[2];
    T g, wall_u[2];
    T kq[2][9];           // K_s(q) = weight_norm (G1_s w_att(q) + G2_s w_rep(q)) by shell q
    T kc[3];              // weight_norm G_AB w_cross(q), q = 1, 2 (zero for one species)
};

template <typename T>
__device__ __forceinline__ T psi3(const Step3<T>& C, int s, T rho);
template <>
__device__ __forceinline__ float psi3<float>(const Step3<float>& C, int s, float rho) {
    return C.psi_form == 1 ? rho : 1.0f - __expf(-rho * C.inv_rho0[s]);
}
template <>
__device__ __forceinline__ double psi3<double>(const Step3<double>& C, int s, double rho) {
    return C.psi_form == 1 ? rho : 1.0 - exp(-rho / C.rho0[s]);
}

__device__ __forceinline__ int wrap3(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}
// reflection about the walls at -1/2 and n - 1/2 (the mirror reading of the ghost rows)
__device__ __forceinline__ int mirror3(int i, int n) {
    int m = i % (2 * n);
    if (m < 0) m += 2 * n;
    return m >= n ? 2 * n - 1 - m : m;
}

// The step's two kernels are launched with programmatic dependent launch: the next kernel's CTAs
// may be scheduled while this grid drains, and every thread waits for the previous grid in the
// stream (and the visibility of its writes) before its first global access.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

template <typename... K, typename... A>
cudaError_t launch_pdl(void (*kernel)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<A&&>(args)...);
}

// ---- k3_density --------------------------------------------------------------------------

// The padded coordinates (own, then ghosts) that hold the value of coordinate v of an axis of
// n sites with g ghosts on each side: periodic images, or the mirror images with `mirror`.
__device__ __forceinline__ int ghost_list(int v, int n, int g, bool mirror, int* out) {
    int k = 0;
    out[k++] = v + g;
    if (v >= g && v < n - g) return k;
    for (int q = -g; q < n + g; ++q) {
        if (q >= 0 && q < n) {
            q = n - 1;  // skip the interior
            continue;
        }
        const int src = mirror ? mirror3(q, n) : wrap3(q, n);
        if (src == v && k < 2 * g + 1) out[k++] = q + g;
    }
    return k;
}

// The density pass: each site's sums over its 19 populations per species give rho_s and psi_s,
// written with their ghost images into the two volumes.  One thread per site: x from the block
// (128 sites of a row), y and z from the grid, looping when the grid is smaller than the lattice
// (the plain pass launches one block per row segment, so each loop runs once).  TOT: the block's
// FP64 partials of the totals of the state go to part[block] as well -- the sums over its sites of
// each species' density deviation sum_l f_l and of the lattice momentum: a site's sums (its two
// species' momenta added) in the context's precision, the sums over the sites in FP64 (the
// FP64 pipe is the scarce one), in a fixed order.
// 16 CTAs per SM for the plain FP32 pass (32 registers, as it ran fastest); 8 with the totals,
// whose FP64 accumulators need up to 64 registers, and in FP64, so that neither spills
template <typename T, bool TOT>
__global__ void __launch_bounds__(128, TOT || sizeof(T) == 8 ? 8 : 16)
    k3_density(const T* __restrict__ f, T* __restrict__ vol, const Step3<T> C, double* __restrict__ part) {
    using V = typename PairOf<T>::V;
    pdl_enter();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    double mass0 = 0.0, mass1 = 0.0, momx = 0.0, momy = 0.0, momz = 0.0;
    V* const P = reinterpret_cast<V*>(vol);
    for (int z = blockIdx.z; z < C.nz; z += gridDim.z)
        for (int y = blockIdx.y; y < C.ny; y += gridDim.y) {
            if (x >= C.nx) continue;
            const long long i = ((long long)z * C.ny + y) * C.pitch + x;
            T rho[2] = {T(0), T(0)}, psi[2] = {T(0), T(0)};
            T mx = T(0), my = T(0), mz = T(0);
#pragma unroll
            for (int s = 0; s < 2; ++s) {  // unrolled, so that the per-species values stay in registers
                if (s >= C.ns) break;
                T a = T(0);
#pragma unroll
                for (int l = 0; l < 19; ++l) {
                    const T v = f[(s * 19 + l) * C.plane + i];
                    a += v;
                    if constexpr (TOT) {
                        if (c3x(l)) mx += c3x(l) > 0 ? v : -v;
                        if (c3y(l)) my += c3y(l) > 0 ? v : -v;
                        if (c3z(l)) mz += c3z(l) > 0 ? v : -v;
                    }
                }
                rho[s] = C.rho_ref[s] + a;
                psi[s] = psi3<T>(C, s, rho[s]);
                if constexpr (TOT) {
                    if (s == 0)
                        mass0 += (double)a;
                    else
                        mass1 += (double)a;
                }
            }
            if constexpr (TOT) {
                momx += (double)mx;
                momy += (double)my;
                momz += (double)mz;
            }
            V pv, rv;
            pv.x = psi[0];
            pv.y = psi[1];
            rv.x = rho[0];
            rv.y = rho[1];
            int xs[2 * GX + 1], ys[2 * GY + 1], zs[2 * GZ + 1];
            const int nxl = ghost_list(x, C.nx, GX, false, xs);
            const int nyl = ghost_list(y, C.ny, GY, false, ys);
            const int nzl = ghost_list(z, C.nz, GZ, C.zbc != 0, zs);
            for (int c = 0; c < nzl; ++c)
                for (int b = 0; b < nyl; ++b)
                    for (int a = 0; a < nxl; ++a) {
                        const long long o = ((long long)zs[c] * C.gy + ys[b]) * C.gpitch + xs[a];
                        P[o] = pv;
                        P[C.gvol + o] = rv;
                    }
        }
    if constexpr (TOT) {
        __shared__ double red[5][128];
        red[0][threadIdx.x] = mass0;
        red[1][threadIdx.x] = mass1;
        red[2][threadIdx.x] = momx;
        red[3][threadIdx.x] = momy;
        red[4][threadIdx.x] = momz;
        __syncthreads();
        for (int h = 64; h > 0; h >>= 1) {
            if ((int)threadIdx.x < h)
                for (int q = 0; q < 5; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h];
            __syncthreads();
        }
        const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        if (threadIdx.x < 5) part[blk * 5 + threadIdx.x] = red[threadIdx.x][0];
    }
}

// out = mass A, mass B, momentum x, y, z: the sum of part[b][q] over the nblk blocks (thread t adds
// blocks t, t + 256, ... in order, then a fixed tree over the threads; FP64, the same bits on every
// call), plus base[q] (the sites times rho_ref,s for the masses).
__global__ void __launch_bounds__(256)
    k3_totals_sum(const double* __restrict__ part, int nblk, double base0, double base1, double* __restrict__ out) {
    __shared__ double red[5][256];
    double a[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblk; b += 256)
        for (int q = 0; q < 5; ++q) a[q] += part[b * 5 + q];
    for (int q = 0; q < 5; ++q) red[q][threadIdx.x] = a[q];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int q = 0; q < 5; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 5) {
        const double base = threadIdx.x == 0 ? base0 : (threadIdx.x == 1 ? base1 : 0.0);
        out[threadIdx.x] = red[threadIdx.x][0] + base;
    }
}

// ---- k3_step -----------------------------------------------------------------------------

enum { K3_WRITE = 1, K3_FIELDS = 2 };

template <typename T, int TY, int TZ>
struct Smem3 {
    static constexpr int BY = TY + 2 * GY, BZ = TZ + 2 * GZ;
    typename PairOf<T>::V box[2][BZ][BY][BX];  // psi, rho pairs of the tile and its halo
    alignas(8) unsigned long long bar;
};

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// The links of Eq. FORCE, one of each antipodal pair (first nonzero component positive), by
// shell |c|^2 = 1, 2, 3, 4, 5, 6, 8.
#define LBM3_SHELL1(L) L(0, 0, 1) L(0, 1, 0) L(1, 0, 0)
#define LBM3_SHELL2(L) L(0, 1, -1) L(0, 1, 1) L(1, -1, 0) L(1, 0, -1) L(1, 0, 1) L(1, 1, 0)
#define LBM3_SHELL3(L) L(1, -1, -1) L(1, -1, 1) L(1, 1, -1) L(1, 1, 1)
#define LBM3_SHELL4(L) L(0, 0, 2) L(0, 2, 0) L(2, 0, 0)
#define LBM3_SHELL5(L)                                                                                      \
    L(0, 1, -2) L(0, 1, 2) L(0, 2, -1) L(0, 2, 1) L(1, -2, 0) L(1, 0, -2) L(1, 0, 2) L(1, 2, 0) L(2, -1, 0) \
        L(2, 0, -1) L(2, 0, 1) L(2, 1, 0)
#define LBM3_SHELL6(L)                                                                                    \
    L(1, -2, -1) L(1, -2, 1) L(1, -1, -2) L(1, -1, 2) L(1, 1, -2) L(1, 1, 2) L(1, 2, -1) L(1, 2, 1)       \
        L(2, -1, -1) L(2, -1, 1) L(2, 1, -1) L(2, 1, 1)
#define LBM3_SHELL8(L) L(0, 2, -2) L(0, 2, 2) L(2, -2, 0) L(2, 0, -2) L(2, 0, 2) L(2, 2, 0)

// c * d added into an accumulator for a constant component c in -2..2
template <int C, typename V>
__device__ __forceinline__ V addc(V acc, V d) {
    if constexpr (C == 1) return vadd(acc, d);
    if constexpr (C == -1) return vsub(acc, d);
    if constexpr (C == 2 || C == -2) return vfma(vsplat(decltype(d.x)(C)), d, acc);
    return acc;
}

// Eq. FORCE over the 46 antipodal link pairs, shell by shell, both species at once, and the cross
// repulsion of Sec. IV over the first belt: F[s][axis] of the site whose psi and rho pairs at the
// offset (dx, dy, dz) are ps(dx, dy, dz) and rh(dx, dy, dz).
template <typename T, int NS, typename PSF, typename RHF>
__device__ __forceinline__ void force3(const Step3<T>& C, const PSF& ps, const RHF& rh, T (&F)[2][3]) {
    using V = typename PairOf<T>::V;
#define PS(dx, dy, dz) ps(dx, dy, dz)
#define RH(dx, dy, dz) rh(dx, dy, dz)
    const V zero = vsplat(T(0));
    V ax = zero, ay = zero, az = zero;
#define LBM3_ACC(dx, dy, dz)                                \
    {                                                       \
        const V d_ = vsub(PS(dx, dy, dz), PS(-(dx), -(dy), -(dz))); \
        sx = addc<dx>(sx, d_);                              \
        sy = addc<dy>(sy, d_);                              \
        sz = addc<dz>(sz, d_);                              \
    }
#define LBM3_SHELL(q, LIST)                          \
    {                                                \
        V sx = zero, sy = zero, sz = zero;           \
        LIST(LBM3_ACC)                               \
        V kq_;                                       \
        kq_.x = C.kq[0][q];                          \
        kq_.y = C.kq[1][q];                          \
        ax = vfma(kq_, sx, ax);                      \
        ay = vfma(kq_, sy, ay);                      \
        az = vfma(kq_, sz, az);                      \
    }
    LBM3_SHELL(1, LBM3_SHELL1)
    LBM3_SHELL(2, LBM3_SHELL2)
    LBM3_SHELL(3, LBM3_SHELL3)
    LBM3_SHELL(4, LBM3_SHELL4)
    LBM3_SHELL(5, LBM3_SHELL5)
    LBM3_SHELL(6, LBM3_SHELL6)
    LBM3_SHELL(8, LBM3_SHELL8)
#undef LBM3_SHELL
#undef LBM3_ACC
    const V p0 = PS(0, 0, 0), r0 = RH(0, 0, 0);
    const V mp = vsub(zero, p0);
    V Fx = vmul(mp, ax), Fy = vmul(mp, ay), Fz = vmul(mp, az);
    if constexpr (NS == 2) {
        // cross repulsion: F_s += -G_AB rho_s(x) sum_l w(|c|^2) rho_s'(x + c_l) c_l over the first belt
        V bx1 = zero, by1 = zero, bz1 = zero, bx2 = zero, by2 = zero, bz2 = zero;
#define LBM3_XACC(dx, dy, dz, SX, SY, SZ)                      \
    {                                                          \
        const V d_ = vsub(RH(dx, dy, dz), RH(-(dx), -(dy), -(dz)));  \
        SX = addc<dx>(SX, d_);                                 \
        SY = addc<dy>(SY, d_);                                 \
        SZ = addc<dz>(SZ, d_);                                 \
    }
#define LBM3_X1(dx, dy, dz) LBM3_XACC(dx, dy, dz, bx1, by1, bz1)
#define LBM3_X2(dx, dy, dz) LBM3_XACC(dx, dy, dz, bx2, by2, bz2)
        LBM3_SHELL1(LBM3_X1)
        LBM3_SHELL2(LBM3_X2)
#undef LBM3_X1
#undef LBM3_X2
#undef LBM3_XACC
        const V k1 = vsplat(C.kc[1]), k2 = vsplat(C.kc[2]);
        const V cx_ = vfma(k2, bx2, vmul(k1, bx1)), cy_ = vfma(k2, by2, vmul(k1, by1)),
                cz_ = vfma(k2, bz2, vmul(k1, bz1));
        const V mr = vsub(zero, r0);
        // species A sees the sums over rho_B, species B those over rho_A
        Fx = vfma(mr, vswap(cx_), Fx);
        Fy = vfma(mr, vswap(cy_), Fy);
        Fz = vfma(mr, vswap(cz_), Fz);
    }
    F[0][0] = Fx.x;
    F[0][1] = Fy.x;
    F[0][2] = Fz.x;
    F[1][0] = Fx.y;
    F[1][1] = Fy.y;
    F[1][2] = Fz.y;
#undef PS
#undef RH
}

// The moments of the site's populations f, the body force along x, the common velocity of R5;
// then (K3_FIELDS) rho_s, u and the plain populations into `fields`, or (K3_WRITE) the
// shifted-velocity BGK of Sec. II and the push of the new populations to x + c_l.  Every scalar
// operation has its rounding fixed (smul, sadd, sfma), so a kernel that inlines this computes the
// same bits whatever the code around it.
template <typename T, int NS, int MODE>
__device__ __forceinline__ void site3(const Step3<T>& C, const T (&f)[NS][19], T (&F)[2][3], int x, int y, int z,
                                      long long i, T* __restrict__ fout, int* __restrict__ flag,
                                      double* __restrict__ fields) {
    using V = typename PairOf<T>::V;
    // ---- moments, body force, common velocity ----
    T rho[NS], ir[NS], jx[NS], jy[NS], jz[NS], drho[NS];
    bool bad = false;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        // each sum starts from its first term (no add of zero)
        T a = f[s][0], mx = f[s][first19(0)], my = f[s][first19(1)], mz = f[s][first19(2)];
#pragma unroll
        for (int l = 1; l < 19; ++l) {
            a = sadd(a, f[s][l]);
            if (c3x(l) && l != first19(0)) mx = sadd(mx, c3x(l) > 0 ? f[s][l] : -f[s][l]);
            if (c3y(l) && l != first19(1)) my = sadd(my, c3y(l) > 0 ? f[s][l] : -f[s][l]);
            if (c3z(l) && l != first19(2)) mz = sadd(mz, c3z(l) > 0 ? f[s][l] : -f[s][l]);
        }
        drho[s] = a;
        rho[s] = sadd(C.rho_ref[s], a);
        if (!(rho[s] > T(0)) || !(rho[s] < T(1e30))) bad = true;
        ir[s] = T(1) / rho[s];
        jx[s] = mx;
        jy[s] = my;
        jz[s] = mz;
        F[s][0] = sfma(rho[s], C.g, F[s][0]);
    }
    if (bad) atomicOr(flag, 1);
    T nxu = T(0), nyu = T(0), nzu = T(0), den = T(0);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        nxu = sfma(C.omega[s], jx[s], nxu);
        nyu = sfma(C.omega[s], jy[s], nyu);
        nzu = sfma(C.omega[s], jz[s], nzu);
        den = sfma(C.omega[s], rho[s], den);
    }
    const T iden = T(1) / den;
    const T upx = smul(nxu, iden), upy = smul(nyu, iden), upz = smul(nzu, iden);

    if constexpr ((MODE & K3_FIELDS) != 0) {
        // rho_s, the barycentric velocity (sum_s j_s + F_s / 2) / sum_s rho_s, plain populations
        const long long n = (long long)C.nx * C.ny * C.nz, k = ((long long)z * C.ny + y) * C.nx + x;
        T mxs = T(0), mys = T(0), mzs = T(0), rt = T(0);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            mxs += jx[s] + T(0.5) * F[s][0];
            mys += jy[s] + T(0.5) * F[s][1];
            mzs += jz[s] + T(0.5) * F[s][2];
            rt += rho[s];
            fields[s * n + k] = (double)rho[s];
#pragma unroll
            for (int l = 0; l < 19; ++l)
                fields[(NS + 3 + s * 19 + l) * n + k] = (double)f[s][l] + w19<double>(l) * (double)C.rho_ref[s];
        }
        fields[(NS + 0) * n + k] = (double)(mxs / rt);
        fields[(NS + 1) * n + k] = (double)(mys / rt);
        fields[(NS + 2) * n + k] = (double)(mzs / rt);
    }

    if constexpr ((MODE & K3_WRITE) != 0) {
        // ---- shifted-velocity BGK (Sec. II) and streaming ----
        // Destinations: the site's index plus one offset per axis, chosen by the sign of c_l; the
        // periodic wrap is folded into those offsets once per thread (walls in z are handled by
        // bounce-back below).
        const long long row = C.pitch, lay = (long long)C.ny * C.pitch;
        const bool wall_lo = C.zbc && z == 0, wall_hi = C.zbc && z == C.nz - 1;
        // FP32: the wrapped offsets of each axis precomputed; FP64 (short of registers): the
        // destination of each population wrapped where it is stored
        long long oxm = 0, oxp = 0, oym = 0, oyp = 0, ozm = 0, ozp = 0;
        if constexpr (sizeof(T) == 4) {
            oxm = x == 0 ? C.nx - 1 : -1;
            oxp = x == C.nx - 1 ? -(C.nx - 1) : 1;
            oym = y == 0 ? (C.ny - 1) * row : -row;
            oyp = y == C.ny - 1 ? -(C.ny - 1) * row : row;
            ozm = z == 0 ? (C.nz - 1) * lay : -lay;
            ozp = z == C.nz - 1 ? -(C.nz - 1) * lay : lay;
        }
        auto push = [&](int s, int l, T v) {
            const int cx_ = c3x(l), cy_ = c3y(l), cz_ = c3z(l);
            if ((cz_ < 0 && wall_lo) || (cz_ > 0 && wall_hi)) {  // halfway bounce-back with Ladd's term
                const T uw = cz_ < 0 ? C.wall_u[0] : C.wall_u[1];
                fout[(s * 19 + opp19(l)) * C.plane + i] = sadd(v, -smul(smul(T(6 * cx_) * w19<T>(l), rho[s]), uw));
                return;
            }
            if constexpr (sizeof(T) == 4) {
                const long long o = (cx_ < 0 ? oxm : (cx_ > 0 ? oxp : 0)) + (cy_ < 0 ? oym : (cy_ > 0 ? oyp : 0)) +
                                    (cz_ < 0 ? ozm : (cz_ > 0 ? ozp : 0));
                fout[(s * 19 + l) * C.plane + i + o] = v;
            } else {
                int xd = x + cx_, yd = y + cy_, zd = z + cz_;
                xd = xd < 0 ? xd + C.nx : (xd >= C.nx ? xd - C.nx : xd);
                yd = yd < 0 ? yd + C.ny : (yd >= C.ny ? yd - C.ny : yd);
                zd = zd < 0 ? zd + C.nz : (zd >= C.nz ? zd - C.nz : zd);
                fout[(s * 19 + l) * C.plane + ((long long)zd * C.ny + yd) * C.pitch + xd] = v;
            }
        };
        if constexpr (NS == 2 && sizeof(T) == 4) {
            // both species in lockstep, (A, B) pairs of packed FP32 instructions
            V fp[19];
#pragma unroll
            for (int l = 0; l < 19; ++l) {
                fp[l].x = f[0][l];
                fp[l].y = f[1][l];
            }
            V rh, drh, om, tau, fx, fy, fz;
            rh.x = rho[0], rh.y = rho[1];
            drh.x = drho[0], drh.y = drho[1];
            om.x = C.omega[0], om.y = C.omega[1];
            tau.x = smul(C.tau[0], ir[0]), tau.y = smul(C.tau[1], ir[1]);
            fx.x = F[0][0], fx.y = F[1][0];
            fy.x = F[0][1], fy.y = F[1][1];
            fz.x = F[0][2], fz.y = F[1][2];
            const V keep = vsub(vsplat(T(1)), om);
            const V ux = vfma(fx, tau, vsplat(upx)), uy = vfma(fy, tau, vsplat(upy)), uz = vfma(fz, tau, vsplat(upz));
            const V u15 = vmul(vsplat(T(1.5)), vfma(ux, ux, vfma(uy, uy, vmul(uz, uz))));
            const V b = vmul(om, rh);
            const V base = vsub(vmul(om, drh), vmul(b, u15));  // omega (drho - 3/2 rho u^2)
            push(0, 0, vfma(keep, fp[0], vmul(vsplat(w19<T>(0)), base)).x);
            push(1, 0, vfma(keep, fp[0], vmul(vsplat(w19<T>(0)), base)).y);
#pragma unroll
            for (int l = 1; l < 19; l += 2) {  // l and its opposite l + 1
                // c_l . u with the components +-1 or 0 of this l (the branches fold away unrolled)
                // from zero: starting from the first component, as the scalar path does, saves an
                // add but changed the register allocation of this build for the worse (measured)
                V cu = vsplat(T(0));
                if (c3x(l) > 0) cu = vadd(cu, ux);
                if (c3x(l) < 0) cu = vsub(cu, ux);
                if (c3y(l) > 0) cu = vadd(cu, uy);
                if (c3y(l) < 0) cu = vsub(cu, uy);
                if (c3z(l) > 0) cu = vadd(cu, uz);
                if (c3z(l) < 0) cu = vsub(cu, uz);
                const T w = w19<T>(l);
                const V wb = vmul(vsplat(w), b);
                const V even = vfma(vmul(vsplat(T(4.5)), wb), vmul(cu, cu), vmul(vsplat(w), base));
                const V odd = vmul(vmul(vsplat(T(3)), wb), cu);
                const V gp = vadd(vfma(keep, fp[l], even), odd);
                const V gm = vsub(vfma(keep, fp[l + 1], even), odd);
                push(0, l, gp.x);
                push(1, l, gp.y);
                push(0, l + 1, gm.x);
                push(1, l + 1, gm.y);
            }
        } else {
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                // the operations of the packed path, one species at a time
                const T om = C.omega[s], keep = T(1) - om, tir = smul(C.tau[s], ir[s]);
                const T ux = sfma(F[s][0], tir, upx), uy = sfma(F[s][1], tir, upy), uz = sfma(F[s][2], tir, upz);
                const T u15 = smul(T(1.5), sfma(ux, ux, sfma(uy, uy, smul(uz, uz))));
                const T b = smul(om, rho[s]);
                const T base = sadd(smul(om, drho[s]), -smul(b, u15));  // omega (drho - 3/2 rho u^2)
                push(s, 0, sfma(keep, f[s][0], smul(w19<T>(0), base)));
#pragma unroll
                for (int l = 1; l < 19; l += 2) {  // l and its opposite l + 1
                    // starting from the first, +1, component (no add of zero)
                    T cu = c3x(l) ? ux : (c3y(l) ? uy : uz);
                    if (c3x(l) && c3y(l)) cu = sadd(cu, c3y(l) > 0 ? uy : -uy);
                    if ((c3x(l) || c3y(l)) && c3z(l)) cu = sadd(cu, c3z(l) > 0 ? uz : -uz);
                    const T w = w19<T>(l);
                    const T wb = smul(w, b);
                    const T even = sfma(smul(T(4.5), wb), smul(cu, cu), smul(w, base));
                    const T odd = smul(smul(T(3), wb), cu);
                    push(s, l, sadd(sfma(keep, f[s][l], even), odd));
                    push(s, l + 1, sadd(sfma(keep, f[s][l + 1], even), -odd));
                }
            }
        }
    }
}

// FP32 tiles of 256 threads: 3 CTAs per SM (80 registers, 16 bytes of spills), measured faster than
// 2 CTAs at 110 registers without spills -- the kernel waits on memory and more warps hide it.
template <typename T, int MODE, int NS, int TY, int TZ>
__global__ void __launch_bounds__(TX* TY* TZ, TX* TY* TZ > 256 ? 1 : (sizeof(T) == 4 ? 3 : 2))
    k3_step(const __grid_constant__ CUtensorMap vmap, const T* __restrict__ fin, T* __restrict__ fout,
            const Step3<T> C, int* __restrict__ flag, double* __restrict__ fields) {
    using V = typename PairOf<T>::V;
    extern __shared__ __align__(1024) unsigned char smem3[];
    Smem3<T, TY, TZ>& S = *reinterpret_cast<Smem3<T, TY, TZ>*>(smem3);
    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    const int tid = (tz * TY + ty) * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
    const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
    const bool live = x < C.nx && y < C.ny && z < C.nz;
    pdl_enter();
    if (tid == 0) {
        const unsigned bar = su32(&S.bar);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        constexpr unsigned bytes = (unsigned)sizeof(S.box);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
        // box origin: padded (x0, y0, z0) = site (x0 - GX, y0 - GY, z0 - GZ); x counts values of T
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
            "%5}], [%6];\n" ::"r"(su32(&S.box[0][0][0][0])),
            "l"(&vmap), "r"(2 * x0), "r"(y0), "r"(z0), "r"(0), "r"(bar)
            : "memory");
    }
    // own populations from HBM while the box is on its way
    const long long i = ((long long)z * C.ny + y) * C.pitch + x;
    T f[NS][19];
    if (live) {
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int l = 0; l < 19; ++l) f[s][l] = fin[(s * 19 + l) * C.plane + i];
    }
    __syncthreads();  // the barrier is initialised before anyone waits on it
    bool ok = true;
    {
        const unsigned bar = su32(&S.bar);
        const long long t0 = clock64();
        for (;;) {
            unsigned done;
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(bar), "r"(0u)
                : "memory");
            if (done) break;
            if (clock64() - t0 > WAIT_LIMIT) {
                ok = false;
                break;
            }
        }
    }
    if (__syncthreads_or(!ok)) {
        if (tid == 0) {
            atomicOr(flag, 2);
            // the copy that did not arrive in time is waited for (bounded) before the CTA exits
            const unsigned bar = su32(&S.bar);
            const long long t0 = clock64();
            for (;;) {
                unsigned done;
                asm volatile(
                    "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, "
                    "p;\n}\n"
                    : "=r"(done)
                    : "r"(bar), "r"(0u)
                    : "memory");
                if (done || clock64() - t0 > WAIT_LIMIT) break;
            }
        }
        return;
    }
    if (!live) return;

    const int bx = tx + GX, by = ty + GY, bz = tz + GZ;
    T F[2][3];
    force3<T, NS>(
        C, [&](int dx, int dy, int dz) { return S.box[0][bz + dz][by + dy][bx + dx]; },
        [&](int dx, int dy, int dz) { return S.box[1][bz + dz][by + dy][bx + dx]; }, F);
    site3<T, NS, MODE>(C, f, F, x, y, z, i, fout, flag, fields);
}

// ---- equilibrium at rest, totals ---------------------------------------------------------------

template <typename T>
__global__ void k3_init(T* __restrict__ f, const double* __restrict__ rho, const Step3<T> C) {
    const long long n = (long long)C.nx * C.ny * C.nz;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % C.nx), y = (int)(k / C.nx % C.ny), z = (int)(k / ((long long)C.nx * C.ny));
        const long long i = ((long long)z * C.ny + y) * C.pitch + x;
        for (int s = 0; s < C.ns; ++s) {
            const double d = rho[s * n + k] - (double)C.rho_ref[s];
            for (int l = 0; l < 19; ++l) f[(s * 19 + l) * C.plane + i] = (T)(w19<double>(l) * d);
        }
    }
}

template <typename T, int MODE, int NS, int TY, int TZ>
cudaError_t launch_step3(const CUtensorMap& map, const T* fin, T* fout, const Step3<T>& C, int* flag, double* fields,
                         cudaStream_t st) {
    const size_t smem = sizeof(Smem3<T, TY, TZ>);
    static bool attr = false;  // per template instance
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(k3_step<T, MODE, NS, TY, TZ>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const dim3 grid((C.nx + TX - 1) / TX, (C.ny + TY - 1) / TY, (C.nz + TZ - 1) / TZ);
    return launch_pdl(k3_step<T, MODE, NS, TY, TZ>, grid, dim3(TX, TY, TZ), smem, st, map, fin, fout, C, flag, fields);
}

template <typename T, int MODE, int NS>
cudaError_t launch_shape(int shape, const CUtensorMap& map, const T* fin, T* fout, const Step3<T>& C, int* flag,
                         double* fields, cudaStream_t st) {
    switch (shape) {
        case 0: return launch_step3<T, MODE, NS, SHAPE_TY[0], SHAPE_TZ[0]>(map, fin, fout, C, flag, fields, st);
        case 1: return launch_step3<T, MODE, NS, SHAPE_TY[1], SHAPE_TZ[1]>(map, fin, fout, C, flag, fields, st);
        case 2: return launch_step3<T, MODE, NS, SHAPE_TY[2], SHAPE_TZ[2]>(map, fin, fout, C, flag, fields, st);
        case 3: return launch_step3<T, MODE, NS, SHAPE_TY[3], SHAPE_TZ[3]>(map, fin, fout, C, flag, fields, st);
        default: return cudaErrorInvalidValue;
    }
}

// the step pass in the chosen tile shape; the fields pass (lbm3_get_fields) in shape 0
template <typename T>
cudaError_t launch_step3_any(int mode, int ns, int shape, const CUtensorMap& map, const T* fin, T* fout,
                             const Step3<T>& C, int* flag, double* fields, cudaStream_t st) {
    if (mode == K3_WRITE)
        return ns == 2 ? launch_shape<T, K3_WRITE, 2>(shape, map, fin, fout, C, flag, fields, st)
                       : launch_shape<T, K3_WRITE, 1>(shape, map, fin, fout, C, flag, fields, st);
    return ns == 2 ? launch_step3<T, K3_FIELDS, 2, SHAPE_TY[0], SHAPE_TZ[0]>(map, fin, fout, C, flag, fields, st)
                   : launch_step3<T, K3_FIELDS, 1, SHAPE_TY[0], SHAPE_TZ[0]>(map, fin, fout, C, flag, fields, st);
}

}  // namespace lbm3

// ---------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------
using namespace lbm3;

struct lbm3_ctx {
    lbm3_desc d{};
    lbm_params p{};
    bool have_params = false, have_fields = false;
    bool own_stream = false;
    cudaStream_t stream = nullptr;
    size_t esize = 4;
    int pitch = 0, gpitch = 0;
    long long plane = 0, gvol = 0, n = 0;
    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    void* vol = nullptr;               // psi and rho volumes: [2][gz][gy][gpitch] pairs
    alignas(64) unsigned char map[NSHAPE][128] = {};  // TMA descriptors of vol, per tile shape
    int shape = 0;                     // tile shape of the step pass (lbm3_autotune)
    int* flag = nullptr;
    double* staging = nullptr;         // lbm3_get_fields / lbm3_set_fields from the host
    size_t staging_bytes = 0;
    double* part = nullptr;            // the density pass's block partials of the totals
    double* tot = nullptr;             // lbm3_totals: the 5 totals on the device
    double* dcheck = nullptr;          // lbm3_set_fields: DCHECK_DOUBLES doubles (launch_density_check)
    int nblk_den = 0;                  // blocks of the density pass with totals
    int tot_grid[3] = {1, 1, 1};       // its grid
    double rho_ref[2] = {0.0, 0.0};
    Step3<float> c32{};
    Step3<double> c64{};
    bool profiling = false;
    std::vector<cudaEvent_t> ev;       // 4 per timed step
    size_t ev_used = 0;
    long long step = 0;
    cudaEvent_t tev[64] = {};          // lbm3_step_totals: an event per ticket (ring)
    long long tickets = 0;             // tickets issued
    std::string err;
};

static std::string g3_create_error;

static int fail3(lbm3_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    else
        g3_create_error = buf;
    return code;
}

#define CK3(call)                                                                                            \
    do {                                                                                                     \
        cudaError_t e_ = (call);                                                                             \
        if (e_ != cudaSuccess)                                                                               \
            return fail3(c, e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s (%s:%d)", #call, \
                         cudaGetErrorString(e_), __FILE__, __LINE__);                                        \
    } while (0)

template <typename T>
static void fill_step3(const lbm3_ctx* c, Step3<T>& C) {
    C = Step3<T>{};
    C.nx = c->d.nx;
    C.ny = c->d.ny;
    C.nz = c->d.nz;
    C.ns = c->d.n_species;
    C.zbc = c->d.z_boundary;
    C.psi_form = c->p.psi_form;
    C.pitch = c->pitch;
    C.gpitch = c->gpitch;
    C.plane = c->plane;
    C.gvol = c->gvol;
    C.gy = c->d.ny + 2 * GY;
    C.gz = c->d.nz + 2 * GZ;
    C.g = (T)c->p.body_force;
    C.wall_u[0] = (T)c->p.wall_u[0];
    C.wall_u[1] = (T)c->p.wall_u[1];
    const double wn = c->p.weight_norm;
    for (int s = 0; s < 2; ++s) {
        const bool on = s < c->d.n_species;
        const int ps = on ? s : 0;
        C.tau[s] = (T)c->p.tau[ps];
        C.omega[s] = (T)(1.0 / c->p.tau[ps]);
        C.rho0[s] = (T)c->p.rho0[ps];
        C.inv_rho0[s] = (T)(1.0 / c->p.rho0[ps]);
        C.rho_ref[s] = on ? (T)c->rho_ref[s] : T(0);
        for (int q = 0; q < 9; ++q)
            C.kq[s][q] = on ? (T)(wn * (c->p.G1[ps] * w_att3(q) + c->p.G2[ps] * w_rep3(q))) : T(0);
    }
    for (int q = 0; q < 3; ++q) C.kc[q] = c->d.n_species == 2 ? (T)(wn * c->p.G_AB * w_cross3(q)) : T(0);
}

static void refresh3(lbm3_ctx* c) {
    fill_step3<float>(c, c->c32);
    fill_step3<double>(c, c->c64);
}

extern "C" void lbm3_default_desc(lbm3_desc* d) {
    if (!d) return;
    *d = lbm3_desc{};
    d->nx = d->ny = d->nz = 64;
    d->n_species = 2;
    d->precision = LBM_FP32;
    d->z_boundary = LBM_PERIODIC;
}

static int check3(lbm3_ctx* c, const lbm3_desc* d) {
    if (!d) return fail3(c, LBM_EINVAL, "desc is NULL");
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || d->nx > 65536 || d->ny > 65535 || d->nz > 65535)
        return fail3(c, LBM_EINVAL, "nx, ny, nz must be >= 1 (nx <= 65536, ny, nz <= 65535)");
    if ((long long)d->nx * d->ny * d->nz > (1LL << 30)) return fail3(c, LBM_EINVAL, "nx * ny * nz > 2^30");
    if (d->n_species != 1 && d->n_species != 2) return fail3(c, LBM_EINVAL, "n_species must be 1 or 2");
    if (d->precision != LBM_FP32 && d->precision != LBM_FP64) return fail3(c, LBM_EINVAL, "bad precision");
    if (d->z_boundary != LBM_PERIODIC && d->z_boundary != LBM_BOUNCEBACK) return fail3(c, LBM_EINVAL, "bad z_boundary");
    if (d->device < 0) return fail3(c, LBM_EINVAL, "device < 0");
    return LBM_OK;
}

static void release3(lbm3_ctx* c) {
    for (int b = 0; b < 2; ++b) cudaFree(c->f[b]);
    cudaFree(c->vol);
    cudaFree(c->flag);
    cudaFree(c->staging);
    cudaFree(c->part);
    cudaFree(c->tot);
    cudaFree(c->dcheck);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    for (cudaEvent_t e : c->tev)
        if (e) cudaEventDestroy(e);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

static int make_vol_map(lbm3_ctx* c, int shape) {
    const auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(lbm::tensor_map_encoder());
    if (!encode) return 1;
    const cuuint64_t es = c->esize;
    // dims: values of T along x (two per site), rows, layers, the two volumes
    const cuuint64_t dims[4] = {(cuuint64_t)2 * c->gpitch, (cuuint64_t)(c->d.ny + 2 * GY),
                                (cuuint64_t)(c->d.nz + 2 * GZ), 2};
    const cuuint64_t strides[3] = {(cuuint64_t)2 * c->gpitch * es, (cuuint64_t)2 * c->gpitch * (c->d.ny + 2 * GY) * es,
                                   (cuuint64_t)2 * c->gvol * es};
    const cuuint32_t box[4] = {(cuuint32_t)(2 * BX), (cuuint32_t)(SHAPE_TY[shape] + 2 * GY),
                               (cuuint32_t)(SHAPE_TZ[shape] + 2 * GZ), 2};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode(reinterpret_cast<CUtensorMap*>(c->map[shape]),
                              c->esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
                              c->vol, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : 2;
}

extern "C" int lbm3_create(lbm3_ctx** out, const lbm3_desc* d) {
    if (!out) return fail3(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = check3(nullptr, d);
    if (rc) return rc;
    lbm3_ctx* c = new (std::nothrow) lbm3_ctx();
    if (!c) return fail3(nullptr, LBM_ENOMEM, "host allocation failed");
    c->d = *d;
    lbm_default_params(&c->p);
    auto bail = [&](int code) {
        g3_create_error = c->err;
        release3(c);
        delete c;
        return code;
    };
#define CKC3(call)                                                                                       \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess)                                                                           \
            return bail(fail3(c, e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s", #call, \
                              cudaGetErrorString(e_)));                                                  \
    } while (0)
    CKC3(cudaSetDevice(d->device));
    if (d->stream) {
        c->stream = static_cast<cudaStream_t>(d->stream);
    } else {
        CKC3(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    const int nx = d->nx, ny = d->ny, nz = d->nz, ns = d->n_species;
    c->esize = d->precision == LBM_FP64 ? 8 : 4;
    c->pitch = (nx + 31) / 32 * 32;
    c->plane = (long long)nz * ny * c->pitch;
    c->gpitch = (nx + 2 * GX + 3) / 4 * 4;
    c->gvol = (long long)(nz + 2 * GZ) * (ny + 2 * GY) * c->gpitch;
    c->n = (long long)nx * ny * nz;
    const size_t fbytes = (size_t)ns * 19 * c->plane * c->esize;
    for (int b = 0; b < 2; ++b) {
        CKC3(cudaMalloc(&c->f[b], fbytes));
        CKC3(cudaMemsetAsync(c->f[b], 0, fbytes, c->stream));
    }
    const size_t vbytes = (size_t)2 * c->gvol * 2 * c->esize;
    CKC3(cudaMalloc(&c->vol, vbytes));
    CKC3(cudaMemsetAsync(c->vol, 0, vbytes, c->stream));
    CKC3(cudaMalloc(&c->flag, sizeof(int)));
    CKC3(cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
    int nsm = 0;
    CKC3(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, d->device));
    {  // the density pass with totals: about 8 CTAs per SM, each looping over its rows
        const int gx = (nx + 127) / 128, target = 8 * nsm;
        const int gy = std::max(1, std::min(ny, target / gx));
        const int gz = std::max(1, std::min(nz, target / (gx * gy)));
        c->tot_grid[0] = gx;
        c->tot_grid[1] = gy;
        c->tot_grid[2] = gz;
        c->nblk_den = gx * gy * gz;
    }
    CKC3(cudaMalloc(&c->part, (size_t)c->nblk_den * 5 * sizeof(double)));
    CKC3(cudaMalloc(&c->tot, 5 * sizeof(double)));
    CKC3(cudaMalloc(&c->dcheck, lbm::DCHECK_DOUBLES * sizeof(double)));
    for (int k = 0; k < NSHAPE; ++k)
        if (make_vol_map(c, k) != 0)
            return bail(fail3(c, LBM_ECUDA, "cuTensorMapEncodeTiled failed for the psi / rho volumes"));
    CKC3(cudaStreamSynchronize(c->stream));
#undef CKC3
    refresh3(c);
    *out = c;
    return LBM_OK;
}

extern "C" void lbm3_destroy(lbm3_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->d.device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    release3(c);
    delete c;
}

extern "C" const char* lbm3_last_error(const lbm3_ctx* c) { return c ? c->err.c_str() : g3_create_error.c_str(); }

extern "C" int lbm3_set_params(lbm3_ctx* c, const lbm_params* p) {
    if (!c) return LBM_EINVAL;
    if (!p) return fail3(c, LBM_EINVAL, "params is NULL");
    if (lbm_validate_params(p, c->d.n_species) != LBM_OK)
        return fail3(c, LBM_EINVAL, "invalid parameters: %s", lbm_last_error(nullptr));
    if (p->weight_preset != LBM_WEIGHTS_PAPER) return fail3(c, LBM_EINVAL, "the 3-D step has the paper's weights only");
    if (p->psi_wall != LBM_WALL_MIRROR) return fail3(c, LBM_EINVAL, "the 3-D step has the mirror wall reading only");
    c->p = *p;
    c->have_params = true;
    refresh3(c);
    return LBM_OK;
}

static int staging3(lbm3_ctx* c, size_t bytes) {
    if (c->staging_bytes >= bytes) return LBM_OK;
    cudaFree(c->staging);
    c->staging = nullptr;
    c->staging_bytes = 0;
    CK3(cudaMalloc(&c->staging, bytes));
    c->staging_bytes = bytes;
    return LBM_OK;
}

extern "C" int lbm3_set_fields(lbm3_ctx* c, const double* rho, int where) {
    if (!c) return LBM_EINVAL;
    if (!rho) return fail3(c, LBM_EINVAL, "rho is NULL");
    if (where != LBM_HOST && where != LBM_DEVICE) return fail3(c, LBM_EINVAL, "where must be LBM_HOST or LBM_DEVICE");
    if (!c->have_params) return fail3(c, LBM_EINVAL, "lbm3_set_params has not been called");
    CK3(cudaSetDevice(c->d.device));
    const int ns = c->d.n_species;
    const long long n = c->n;
    int rc = staging3(c, (size_t)ns * n * sizeof(double));
    if (rc) return rc;
    // the densities into the staging buffer, checked and summed there (the reference densities
    // need the sums on the host: one small read-back)
    CK3(cudaMemcpyAsync(c->staging, rho, (size_t)ns * n * sizeof(double),
                        where == LBM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream));
    CK3(lbm::launch_density_check(c->staging, n, ns, c->dcheck, c->stream));
    double chk[3];
    CK3(cudaMemcpyAsync(chk, c->dcheck, sizeof chk, cudaMemcpyDeviceToHost, c->stream));
    CK3(cudaStreamSynchronize(c->stream));
    unsigned long long bad;
    memcpy(&bad, &chk[2], sizeof bad);
    if (bad != ~0ull) {
        double v = 0.0;
        CK3(cudaMemcpy(&v, c->staging + bad, sizeof v, cudaMemcpyDeviceToHost));
        return fail3(c, LBM_EINVAL, "rho must be > 0 and finite (rho[%d][%lld] = %g)", (int)(bad / n),
                     (long long)(bad % n), v);
    }
    for (int s = 0; s < 2; ++s)
        c->rho_ref[s] = c->d.precision == LBM_FP64 || s >= ns ? 0.0
                                                               : (c->p.rho_ref[s] >= 0.0 ? c->p.rho_ref[s] : chk[s] / n);
    refresh3(c);
    const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
    if (c->d.precision == LBM_FP64)
        lbm3::k3_init<double><<<blocks, 256, 0, c->stream>>>((double*)c->f[0], c->staging, c->c64);
    else
        lbm3::k3_init<float><<<blocks, 256, 0, c->stream>>>((float*)c->f[0], c->staging, c->c32);
    CK3(cudaGetLastError());
    CK3(cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
    CK3(cudaStreamSynchronize(c->stream));
    c->cur = 0;
    c->step = 0;
    c->have_fields = true;
    return LBM_OK;
}

// the density pass over f[cur] into the volumes; totals: its block partials of the totals of
// f[cur] summed into out (5 doubles, device memory) as well
static cudaError_t density3(lbm3_ctx* c, double* totals = nullptr) {
    const dim3 grid = totals ? dim3(c->tot_grid[0], c->tot_grid[1], c->tot_grid[2])
                             : dim3((c->d.nx + 127) / 128, c->d.ny, c->d.nz);
    const dim3 block(128);
    cudaError_t e;
    if (c->d.precision == LBM_FP64)
        e = totals ? launch_pdl(lbm3::k3_density<double, true>, grid, block, 0, c->stream, (const double*)c->f[c->cur],
                                (double*)c->vol, c->c64, c->part)
                   : launch_pdl(lbm3::k3_density<double, false>, grid, block, 0, c->stream,
                                (const double*)c->f[c->cur], (double*)c->vol, c->c64, (double*)nullptr);
    else
        e = totals ? launch_pdl(lbm3::k3_density<float, true>, grid, block, 0, c->stream, (const float*)c->f[c->cur],
                                (float*)c->vol, c->c32, c->part)
                   : launch_pdl(lbm3::k3_density<float, false>, grid, block, 0, c->stream, (const float*)c->f[c->cur],
                                (float*)c->vol, c->c32, (double*)nullptr);
    if (e != cudaSuccess || !totals) return e;
    // the reference densities the FP32 deviations are taken from (zero in FP64, and for an absent
    // species), once per site
    const double n = (double)c->n;
    const double r0 = c->d.precision == LBM_FP64 ? 0.0 : (double)c->c32.rho_ref[0];
    const double r1 = c->d.precision == LBM_FP64 ? 0.0 : (double)c->c32.rho_ref[1];
    lbm3::k3_totals_sum<<<1, 256, 0, c->stream>>>(c->part, c->nblk_den, n * r0, n * r1, totals);
    return cudaGetLastError();
}

static cudaError_t collide3(lbm3_ctx* c, int mode, double* fields) {
    const int shape = mode == K3_WRITE ? c->shape : 0;
    const CUtensorMap& map = *reinterpret_cast<const CUtensorMap*>(c->map[shape]);
    if (c->d.precision == LBM_FP64)
        return launch_step3_any<double>(mode, c->d.n_species, shape, map, (const double*)c->f[c->cur],
                                        (double*)c->f[c->cur ^ 1], c->c64, c->flag, fields, c->stream);
    return launch_step3_any<float>(mode, c->d.n_species, shape, map, (const float*)c->f[c->cur],
                                   (float*)c->f[c->cur ^ 1], c->c32, c->flag, fields, c->stream);
}

// one step: the density pass and the collide pass (bracketed by events while profiling)
static int one_step3(lbm3_ctx* c) {
    cudaEvent_t* e = nullptr;
    if (c->profiling) {
        if (c->ev_used + 4 > c->ev.size())
            for (int q = 0; q < 64; ++q) {
                cudaEvent_t ev;
                CK3(cudaEventCreate(&ev));
                c->ev.push_back(ev);
            }
        e = &c->ev[c->ev_used];
        c->ev_used += 4;
        CK3(cudaEventRecord(e[0], c->stream));
    }
    CK3(density3(c));
    if (e) {
        CK3(cudaEventRecord(e[1], c->stream));
        CK3(cudaEventRecord(e[2], c->stream));
    }
    CK3(collide3(c, K3_WRITE, nullptr));
    if (e) CK3(cudaEventRecord(e[3], c->stream));
    c->cur ^= 1;
    c->step += 1;
    return LBM_OK;
}

extern "C" int lbm3_step(lbm3_ctx* c, int nsteps) {
    if (!c || nsteps < 0) return c ? fail3(c, LBM_EINVAL, "nsteps < 0") : LBM_EINVAL;
    if (!c->have_fields) return fail3(c, LBM_EINVAL, "lbm3_set_fields has not been called");
    CK3(cudaSetDevice(c->d.device));
    for (int k = 0; k < nsteps; ++k) {
        const int rc = one_step3(c);
        if (rc != LBM_OK) return rc;
    }
    return LBM_OK;
}

extern "C" int lbm3_step_totals(lbm3_ctx* c, int nsteps, double* dst, long long stride, long long* ticket) {
    if (!c) return LBM_EINVAL;
    if (nsteps < 0) return fail3(c, LBM_EINVAL, "nsteps < 0");
    if (!dst && nsteps > 0) return fail3(c, LBM_EINVAL, "dst is NULL");
    if (stride < 5 * (long long)sizeof(double) || stride % (long long)sizeof(double))
        return fail3(c, LBM_EINVAL, "stride must be a multiple of 8 bytes and at least 40");
    if (!c->have_fields) return fail3(c, LBM_EINVAL, "lbm3_set_fields has not been called");
    CK3(cudaSetDevice(c->d.device));
    // the kernels write the records themselves: device memory, or pinned host memory through its
    // device address
    double* out = nullptr;
    if (nsteps > 0) {
        cudaPointerAttributes pa{};
        const cudaError_t e = cudaPointerGetAttributes(&pa, dst);
        cudaGetLastError();  // an unregistered pointer may leave an error behind
        if (e == cudaSuccess && pa.type == cudaMemoryTypeDevice)
            out = dst;
        else if (e == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer)
            out = static_cast<double*>(pa.devicePointer);
        else
            return fail3(c, LBM_EINVAL, "dst must be device memory or pinned host memory");
    }
    // after each collide pass, the density pass of the next step forms the totals of the new state
    // too (so the populations are read once per step for both); the first step needs its own
    for (int k = 0; k < nsteps; ++k) {
        if (k == 0) CK3(density3(c));
        CK3(collide3(c, K3_WRITE, nullptr));
        c->cur ^= 1;
        c->step += 1;
        CK3(density3(c, out + (long long)k * (stride / (long long)sizeof(double))));
    }
    if (nsteps > 0) {  // one event for the run: its last record
        cudaEvent_t& e = c->tev[c->tickets % 64];
        if (!e) CK3(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        CK3(cudaEventRecord(e, c->stream));
        if (ticket) *ticket = c->tickets;
        c->tickets += 1;
    }
    return LBM_OK;
}

extern "C" int lbm3_wait(lbm3_ctx* c, long long ticket) {
    if (!c) return LBM_EINVAL;
    if (ticket < 0 || ticket >= c->tickets) return fail3(c, LBM_EINVAL, "ticket %lld was not issued", ticket);
    CK3(cudaSetDevice(c->d.device));
    if (ticket < c->tickets - 64)
        CK3(cudaStreamSynchronize(c->stream));  // its event was reused: wait for everything
    else
        CK3(cudaEventSynchronize(c->tev[ticket % 64]));
    return LBM_OK;
}

extern "C" int lbm3_synchronize(lbm3_ctx* c) {
    if (!c) return LBM_EINVAL;
    CK3(cudaSetDevice(c->d.device));
    CK3(cudaStreamSynchronize(c->stream));
    int flag = 0;
    CK3(cudaMemcpy(&flag, c->flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag & 2) return fail3(c, LBM_ETIMEOUT, "a bounded device-side wait for a tile load gave up");
    if (flag & 1) return fail3(c, LBM_ENONFINITE, "a step met a density <= 0, NaN or Inf");
    return LBM_OK;
}

extern "C" int lbm3_get_fields(lbm3_ctx* c, double* rho, double* u, double* f, int where) {
    if (!c) return LBM_EINVAL;
    if (where != LBM_HOST && where != LBM_DEVICE) return fail3(c, LBM_EINVAL, "where must be LBM_HOST or LBM_DEVICE");
    if (!c->have_fields) return fail3(c, LBM_EINVAL, "lbm3_set_fields has not been called");
    CK3(cudaSetDevice(c->d.device));
    const int ns = c->d.n_species;
    const long long n = c->n;
    const size_t per = (size_t)(ns + 3 + 19 * ns);
    int rc = staging3(c, per * n * sizeof(double));
    if (rc) return rc;
    CK3(density3(c));
    CK3(collide3(c, K3_FIELDS, c->staging));
    const cudaMemcpyKind kind = where == LBM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (rho) CK3(cudaMemcpyAsync(rho, c->staging, (size_t)ns * n * sizeof(double), kind, c->stream));
    if (u) CK3(cudaMemcpyAsync(u, c->staging + (size_t)ns * n, (size_t)3 * n * sizeof(double), kind, c->stream));
    if (f)
        CK3(cudaMemcpyAsync(f, c->staging + (size_t)(ns + 3) * n, (size_t)19 * ns * n * sizeof(double), kind,
                            c->stream));
    return lbm3_synchronize(c);
}

extern "C" int lbm3_totals(lbm3_ctx* c, double* mass, double* momentum) {
    if (!c) return LBM_EINVAL;
    if (!c->have_fields) return fail3(c, LBM_EINVAL, "lbm3_set_fields has not been called");
    CK3(cudaSetDevice(c->d.device));
    CK3(density3(c, c->tot));  // the density pass with the totals of f[cur]
    double t[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    CK3(cudaMemcpyAsync(t, c->tot, sizeof t, cudaMemcpyDeviceToHost, c->stream));
    const int rc = lbm3_synchronize(c);
    if (rc) return rc;
    if (mass)
        for (int s = 0; s < c->d.n_species; ++s) mass[s] = t[s];
    if (momentum)
        for (int q = 0; q < 3; ++q) momentum[q] = t[2 + q];
    return LBM_OK;
}

extern "C" int lbm3_profile(lbm3_ctx* c, int enable) {
    if (!c) return LBM_EINVAL;
    CK3(cudaSetDevice(c->d.device));
    CK3(cudaStreamSynchronize(c->stream));
    c->profiling = enable != 0;
    c->ev_used = 0;
    return LBM_OK;
}

extern "C" int lbm3_profile_read(lbm3_ctx* c, double* ms, long long* steps) {
    if (!c) return LBM_EINVAL;
    CK3(cudaSetDevice(c->d.device));
    CK3(cudaStreamSynchronize(c->stream));
    double t[2] = {0.0, 0.0};
    for (size_t k = 0; k + 3 < c->ev_used; k += 4)
        for (int j = 0; j < 2; ++j) {
            float v = 0.f;
            CK3(cudaEventElapsedTime(&v, c->ev[k + 2 * j], c->ev[k + 2 * j + 1]));
            t[j] += v;
        }
    if (ms) {
        ms[0] = t[0];
        ms[1] = t[1];
    }
    if (steps) *steps = (long long)(c->ev_used / 4);
    return LBM_OK;
}

extern "C" int lbm3_autotune(lbm3_ctx* c, int steps, int* chosen, double* ms) {
    if (!c) return LBM_EINVAL;
    if (steps < 1 || steps > 10000) return fail3(c, LBM_EINVAL, "steps must be in 1 .. 10000");
    if (!c->have_fields) return fail3(c, LBM_EINVAL, "lbm3_set_fields has not been called");
    CK3(cudaSetDevice(c->d.device));
    // the state is kept aside and put back: the shapes change the schedule, not the arithmetic
    const size_t fbytes = (size_t)c->d.n_species * 19 * c->plane * c->esize;
    void* saved = nullptr;
    CK3(cudaMalloc(&saved, fbytes));
    cudaError_t e = cudaMemcpyAsync(saved, c->f[c->cur], fbytes, cudaMemcpyDeviceToDevice, c->stream);
    const int cur0 = c->cur, shape0 = c->shape;
    const long long step0 = c->step;
    cudaEvent_t a = nullptr, b = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    double t[NSHAPE] = {0.0, 0.0, 0.0, 0.0};
    int best = 0;
    for (int k = 0; k < NSHAPE && e == cudaSuccess; ++k) {
        c->shape = k;
        e = collide3(c, K3_WRITE, nullptr);  // one untimed pass (module load, caches)
        if (e == cudaSuccess) e = cudaEventRecord(a, c->stream);
        for (int i = 0; i < steps && e == cudaSuccess; ++i) {
            e = density3(c);
            if (e == cudaSuccess) e = collide3(c, K3_WRITE, nullptr);
            c->cur ^= 1;
        }
        if (e == cudaSuccess) e = cudaEventRecord(b, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float v = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&v, a, b);
        t[k] = (double)v / steps;
        if (t[k] < t[best]) best = k;
        c->cur = cur0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->f[c->cur], saved, fbytes, cudaMemcpyDeviceToDevice, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(saved);
    c->cur = cur0;
    c->step = step0;
    c->shape = e == cudaSuccess ? best : shape0;
    CK3(e);
    CK3(cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
    if (chosen) *chosen = best;
    if (ms)
        for (int k = 0; k < NSHAPE; ++k) ms[k] = t[k];
    return LBM_OK;
}

extern "C" int lbm3_set_shape(lbm3_ctx* c, int shape) {
    if (!c) return LBM_EINVAL;
    if (shape < 0 || shape >= NSHAPE) return fail3(c, LBM_EINVAL, "shape must be in 0 .. %d", NSHAPE - 1);
    c->shape = shape;
    return LBM_OK;
}
