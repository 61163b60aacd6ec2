#include <cfloat>
// lbm_obs.cu -- initial state, state export and the FP64 reduction of the observables.
#include "lbm_reduce.cuh"

namespace lbm {

namespace {

// Slot of population l of site (x, z) of the lattice whose row -PULL_GZ is padded row prow0 (nz
// rows) in the pull layout: where its gather reads it, at x - c_l, or at (x, opp(l)) when
// x - c_l lies beyond a wall.  Returns the offset within a plane and sets ls to the plane.
// Index i in -n .. 2n - 1 wrapped into 0 .. n - 1 (a neighbour one cell across an edge).
__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

template <typename T>
__device__ long long pull_slot(const StepConst<T>& C, int x, int z, int nz, int prow0, int l, int& ls) {
    const int zs = z - cz(l);
    if (C.zbc && (zs < 0 || zs >= nz)) {
        ls = opp(l);
        return (long long)(prow0 + z + PULL_GZ) * C.pitch + x + PULL_GX;
    }
    ls = l;
    return (long long)(prow0 + wrap1(zs, nz) + PULL_GZ) * C.pitch + wrap1(x - cx(l), C.nx) + PULL_GX;
}

// Populations at the equilibrium of Sec. II for given rho, u (stored as deviations from
// W_l rho_ref; rho_ref = 0 stores plain values).  The arithmetic is done in FP64.  Push layout
// (inst null): the value of (x, l) sits at (x, l).  Pull layout: it sits where the gather of
// (x, l) reads it (pull_slot); every slot is written once.  z runs over the compact rows of all
// lattices of a batch.
// A thread per column x of a row, the rows strided over gridDim.y.  At rest (u null) the
// equilibrium is W_l (rho - rho_ref) exactly, which takes one FP64 product per population.
template <typename T>
__global__ void k_init(int ns, T* __restrict__ f, const double* __restrict__ rho, const double* __restrict__ u,
                       const StepConst<T> C, const InstGeom* __restrict__ inst, int ninst) {
    const long long n = (long long)C.nx * C.nz;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= C.nx) return;
    for (int zg = blockIdx.y; zg < C.nz; zg += gridDim.y) {
        const long long i = (long long)zg * C.nx + x;
        const double ux = u ? u[i] : 0.0, uz = u ? u[n + i] : 0.0;
        int k = 0;
        if (inst && ninst > 1) k = inst_of_row(inst, ninst, zg);
        for (int s = 0; s < ns; ++s) {
            const double r = rho[s * n + i];
            const double dr = r - (double)C.rho_ref[s];
#pragma unroll
            for (int l = 0; l < 9; ++l) {
                long long o = (long long)zg * C.pitch + x;
                int ls = l;
                if (inst) o = pull_slot(C, x, zg - inst[k].zrow0, inst[k].nz, inst[k].prow0, l, ls);
                f[(s * 9 + ls) * C.plane + o] = (T)(u ? feq_dev<double>(l, dr, r, ux, uz) : wlb<double>(l) * dr);
            }
        }
    }
}

// Where the gather of the pull layout reads population l of site (x, z) (as pull_slot), taking
// x - c_l and, without walls, z - c_l from the ghost columns and rows, which hold the periodic
// images of the current state: no wrapping.  For reads only (a write must go to the wrapped slot).
template <typename T>
__device__ __forceinline__ long long pull_src(const StepConst<T>& C, int x, int z, int nz, int prow0, int l, int& ls) {
    const int zs = z - cz(l);
    if (C.zbc && (zs < 0 || zs >= nz)) {
        ls = opp(l);
        return (long long)(prow0 + z + PULL_GZ) * C.pitch + x + PULL_GX;
    }
    ls = l;
    return (long long)(prow0 + zs + PULL_GZ) * C.pitch + (x - cx(l) + PULL_GX);
}

// The post-streaming populations as plain values, [ns][9][nz][nx]: the stored value of (x, l) in
// the push layout, the gather of the pull layout.  Blocks of 32 x 8 sites of one population
// (blockIdx.z = s * 9 + l).
template <typename T, typename O>
__global__ void __launch_bounds__(256) k_export(int ns, const T* __restrict__ f, O* __restrict__ out,
                                                const StepConst<T> C, const InstGeom* __restrict__ inst, int ninst) {
    const long long n = (long long)C.nx * C.nz;
    const int s = blockIdx.z / 9, l = blockIdx.z % 9;
    const int x = blockIdx.x * 32 + threadIdx.x, zg = blockIdx.y * 8 + threadIdx.y;
    if (x >= C.nx || zg >= C.nz) return;
    const double base = wlb<double>(l) * (double)C.rho_ref[s];
    long long o = (long long)zg * C.pitch + x;
    int ls = l;
    if (inst) {
        if (ninst > 1) {
            const int k = inst_of_row(inst, ninst, zg);
            o = pull_src(C, x, zg - inst[k].zrow0, inst[k].nz, inst[k].prow0, l, ls);
        } else {  // one lattice: its rows start at padded row PULL_GZ
            o = pull_src(C, x, zg, C.nz, 0, l, ls);
        }
    }
    out[(s * 9 + l) * n + (long long)zg * C.nx + x] = (O)((double)f[(s * 9 + ls) * C.plane + o] + base);
}

// The inverse of k_export: plain FP64 post-streaming values in, stored values out.
template <typename T>
__global__ void k_import(int ns, T* __restrict__ f, const double* __restrict__ in, const StepConst<T> C,
                         const InstGeom* __restrict__ inst, int ninst) {
    const long long n = (long long)C.nx * C.nz;
    const int s = blockIdx.y / 9, l = blockIdx.y % 9;
    const double base = wlb<double>(l) * (double)C.rho_ref[s];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % C.nx), zg = (int)(i / C.nx);
        long long o = (long long)zg * C.pitch + x;
        int ls = l;
        if (inst) {
            const int k = ninst > 1 ? inst_of_row(inst, ninst, zg) : 0;
            o = pull_slot(C, x, zg - inst[k].zrow0, inst[k].nz, inst[k].prow0, l, ls);
        }
        f[(s * 9 + ls) * C.plane + o] = (T)(in[(s * 9 + l) * n + i] - base);
    }
}

// The reduction kernel: work item blockIdx.x, and with TAIL the last block to finish writes the
// scalar sums into out[O_MASS..] on the device.
template <typename PT, bool TAIL>
__global__ void __launch_bounds__(RB_THREADS) k_reduce(const ObsPtrs O, int nxpart, int nzpart, int nx, int nz, int zbc,
                                                       int nrowblocks, unsigned* ticket, void* __restrict__ out,
                                                       void* __restrict__ avg, void* __restrict__ bpart,
                                                       void* __restrict__ bavg, int accumulate, PT inx, PT inz,
                                                       const InstGeom* __restrict__ inst, int ninst) {
    using R = Red<PT>;
    using A = typename R::A;
    __shared__ A wsc[RB_THREADS / 32][NSC];
    __shared__ A fin[NSC][RB_THREADS];
    __shared__ bool last;
    const int t = threadIdx.x;
    reduce_block<PT>(blockIdx.x, O.part_row, O.part_col, O.flag, nxpart, nzpart, nx, nz, zbc, nrowblocks, out, avg,
                     bpart, bavg, accumulate, inx, inz, wsc, inst, ninst);
    if constexpr (TAIL) {
        // the block's writes happen before thread 0's fence (barrier); the fence is
        // cumulative, so the block drawing the last ticket sees every block's results
        __syncthreads();
        if (t == 0) {
            __threadfence();
            last = atomicAdd(ticket, 1u) == gridDim.x - 1;
            if (last) __threadfence();
        }
        __syncthreads();
        if (!last) return;
        A acc[NSC];
        for (int k = 0; k < NSC; ++k) acc[k] = R::zero();
        for (int b = t; b < (int)gridDim.x; b += RB_THREADS)
            for (int k = 0; k < NSC; ++k) acc[k] = R::add(acc[k], R::get(bpart, (long long)b * NSC + k));
        for (int k = 0; k < NSC; ++k) fin[k][t] = acc[k];
        __syncthreads();
        for (int o = RB_THREADS / 2; o > 0; o >>= 1) {
            if (t < o)
                for (int k = 0; k < NSC; ++k) fin[k][t] = R::add(fin[k][t], fin[k][t + o]);
            __syncthreads();
        }
        if (t == 0) {
            R::put(out, O_MASS, fin[0][0]);
            R::put(out, O_MASS + 1, fin[1][0]);
            R::put(out, O_MOM, fin[2][0]);
            R::put(out, O_MOM + 1, fin[3][0]);
            R::put(out, O_GAMMA, fin[4][0]);
            bool bad = (O.flag[0] & 1) != 0;
            for (int k = 0; k < NSC; ++k) bad = bad || !R::finite(fin[k][0]);
            R::put(out, O_BAD, R::from(bad ? PT(1) : PT(0)));
            if (!zbc) {
                R::put(out, O_WALL, R::zero());
                R::put(out, O_WALL + 1, R::zero());
            }
            *ticket = 0u;
        }
    } else {
        (void)ticket;
        (void)fin;
        (void)last;
    }
}


}  // namespace

// ---- the densities of lbm_set_fields: check and sums -----------------------------------------

// Block b of species blockIdx.y: the values b 256 + t + k 256 DCHECK_BLOCKS, summed per thread in
// that order, then a fixed tree over the block; the first invalid index by atomicMin.
__global__ void __launch_bounds__(256) k_density_check(const double* __restrict__ rho, long long n,
                                                       double* __restrict__ scratch) {
    const int s = blockIdx.y;
    const double* r = rho + s * n;
    double a = 0.0;
    unsigned long long first = ~0ull;
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += 256LL * gridDim.x) {
        const double v = r[i];
        if (!(v > 0.0) || !(v <= DBL_MAX)) first = min(first, (unsigned long long)(s * n + i));  // NaN, <= 0, inf
        a += v;
    }
    if (first != ~0ull) atomicMin(reinterpret_cast<unsigned long long*>(scratch + 2), first);
    __shared__ double red[256];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) scratch[3 + s * gridDim.x + blockIdx.x] = red[0];
}

// scratch[s] = the sum of species s's block sums: thread t adds blocks t, t + 256, ... (one here),
// then a fixed tree.
__global__ void __launch_bounds__(256) k_density_total(int ns, double* __restrict__ scratch) {
    __shared__ double red[256];
    for (int s = 0; s < ns; ++s) {
        double a = 0.0;
        for (int b = threadIdx.x; b < DCHECK_BLOCKS; b += 256) a += scratch[3 + s * DCHECK_BLOCKS + b];
        red[threadIdx.x] = a;
        __syncthreads();
        for (int h = 128; h > 0; h >>= 1) {
            if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) scratch[s] = red[0];
        __syncthreads();
    }
}

cudaError_t launch_density_check(const double* rho, long long n, int ns, double* scratch, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(scratch, 0, 2 * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch + 2, 0xff, sizeof(double), st);
    if (e != cudaSuccess) return e;
    k_density_check<<<dim3(DCHECK_BLOCKS, ns), 256, 0, st>>>(rho, n, scratch);
    k_density_total<<<1, 256, 0, st>>>(ns, scratch);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init(int ns, T* f, const double* rho, const double* u, const StepConst<T>& C, const Batch* B,
                        cudaStream_t st) {
    const dim3 grid((C.nx + 127) / 128, C.nz < 65535 ? C.nz : 65535);
    k_init<T><<<grid, 128, 0, st>>>(ns, f, rho, u, C, B ? B->inst : nullptr, B ? B->ninst : 0);
    return cudaGetLastError();
}

template <typename T, typename O>
cudaError_t launch_export(int ns, const T* f, O* out, const StepConst<T>& C, const Batch* B, cudaStream_t st) {
    const dim3 grid((C.nx + 31) / 32, (C.nz + 7) / 8, 9 * ns);
    k_export<T, O><<<grid, dim3(32, 8), 0, st>>>(ns, f, out, C, B ? B->inst : nullptr, B ? B->ninst : 0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_import(int ns, T* f, const double* in, const StepConst<T>& C, const Batch* B, cudaStream_t st) {
    const long long n = (long long)C.nx * C.nz;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_import<T><<<dim3(blocks, 9 * ns), 256, 0, st>>>(ns, f, in, C, B ? B->inst : nullptr, B ? B->ninst : 0);
    return cudaGetLastError();
}

namespace {
__global__ void k_obs_trailer(double* dst, double samples, long long step, long long averages) {
    dst[0] = samples;
    reinterpret_cast<long long*>(dst)[1] = step;
    reinterpret_cast<long long*>(dst)[2] = averages;
    reinterpret_cast<long long*>(dst)[3] = 0;
}
}  // namespace

cudaError_t launch_obs_trailer(double* dst, double samples, long long step, long long averages, cudaStream_t st) {
    k_obs_trailer<<<1, 1, 0, st>>>(dst, samples, step, averages);
    return cudaGetLastError();
}

namespace {
__global__ void k_snap_check(const unsigned long long* tag, unsigned long long expected, int* flag) {
    if (*tag != expected) atomicOr(flag, 4);
}
}  // namespace

cudaError_t launch_snap_check(const unsigned long long* tag, unsigned long long expected, int* flag,
                              cudaStream_t st) {
    k_snap_check<<<1, 1, 0, st>>>(tag, expected, flag);
    return cudaGetLastError();
}

int reduce_blocks(int nx, int nz) {
    return (nz + RB_THREADS / 32 - 1) / (RB_THREADS / 32) + (nx + RB_THREADS / 32 - 1) / (RB_THREADS / 32);
}

cudaError_t launch_reduce(int precision_bytes, const ObsPtrs& O, int nxpart, int nzpart, int nx, int nz, int zbc,
                          unsigned* ticket, double* out, double* avg, double* bpart, double* bavg, int accumulate,
                          bool tail, const InstGeom* inst, int ninst, cudaStream_t st) {
    const int rb = (nz + RB_THREADS / 32 - 1) / (RB_THREADS / 32);
    const int nb = reduce_blocks(nx, nz);
    if (precision_bytes == 4) {
        if (tail)
            k_reduce<float, true><<<nb, RB_THREADS, 0, st>>>(O, nxpart, nzpart, nx, nz, zbc, rb, ticket, out, avg,
                                                             bpart, bavg, accumulate, 1.0f / nx, 1.0f / nz, inst,
                                                              ninst);
        else
            k_reduce<float, false><<<nb, RB_THREADS, 0, st>>>(O, nxpart, nzpart, nx, nz, zbc, rb, ticket, out, avg,
                                                              bpart, bavg, accumulate, 1.0f / nx, 1.0f / nz, inst,
                                                              ninst);
    } else {
        if (tail)
            k_reduce<double, true><<<nb, RB_THREADS, 0, st>>>(O, nxpart, nzpart, nx, nz, zbc, rb, ticket, out, avg,
                                                              bpart, bavg, accumulate, 1.0 / nx, 1.0 / nz, inst,
                                                               ninst);
        else
            k_reduce<double, false><<<nb, RB_THREADS, 0, st>>>(O, nxpart, nzpart, nx, nz, zbc, rb, ticket, out, avg,
                                                               bpart, bavg, accumulate, 1.0 / nx, 1.0 / nz, inst,
                                                               ninst);
    }
    return cudaGetLastError();
}

template cudaError_t launch_init<float>(int, float*, const double*, const double*, const StepConst<float>&,
                                        const Batch*, cudaStream_t);
template cudaError_t launch_init<double>(int, double*, const double*, const double*, const StepConst<double>&,
                                         const Batch*, cudaStream_t);
template cudaError_t launch_export<float, double>(int, const float*, double*, const StepConst<float>&, const Batch*,
                                                  cudaStream_t);
template cudaError_t launch_export<double, double>(int, const double*, double*, const StepConst<double>&,
                                                   const Batch*, cudaStream_t);
template cudaError_t launch_export<float, float>(int, const float*, float*, const StepConst<float>&, const Batch*,
                                                 cudaStream_t);
template cudaError_t launch_export<double, float>(int, const double*, float*, const StepConst<double>&, const Batch*,
                                                  cudaStream_t);
template cudaError_t launch_import<float>(int, float*, const double*, const StepConst<float>&, const Batch*,
                                          cudaStream_t);
template cudaError_t launch_import<double>(int, double*, const double*, const StepConst<double>&, const Batch*,
                                           cudaStream_t);

}  // namespace lbm
