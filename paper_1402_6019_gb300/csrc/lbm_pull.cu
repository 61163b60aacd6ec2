// lbm_pull.cu -- one-pass time step in the pull layout: persistent CTAs, tiles moved by TMA.
//
// Layout.  The stored value S(x, l) is the post-collision population f*_l(x) of the previous
// step, except that a population leaving x through a wall (x + c_l beyond z = -1/2 or
// z = nz - 1/2) is stored already reflected, S(x, l) = f*_l(x) - 6 W_l rho(x) c_lx U_w (halfway
// bounce-back with Ladd's moving-wall term, Sec. IV): the value that enters x as opp(l) at the
// next step.  The post-streaming populations of Sec. II are then
//     f_l(x) = S(x - c_l, l)          if x - c_l lies in the lattice (x and periodic z wrap),
//     f_l(x) = S(x, opp(l))           if x - c_l lies beyond a wall,
// the same numbers the push layout of the other kernels stores.  Each plane is padded with
// PULL_GX ghost columns on either side and PULL_GZ ghost rows above and below, which hold the
// periodic images of the lattice (rows only without walls); the kernel that writes a boundary
// site also writes its images, so every tile's read is one in-bounds rectangle.
//
// Work.  A CTA of TW x PZ threads (one or two warps per tile row; Shape) loops over tiles.  The populations of
// the tile and of a 3-cell ring around it (2 cells for the psi stencil of Eq. FORCE, 1 more for
// the gather, x rounded to a 16-byte boundary) arrive in shared memory with one 3-D
// cp.async.bulk.tensor load; each warp stores the new populations of its row of 32 sites straight
// from registers, one 128-byte run per plane.  As soon as a tile's box has been read (densities
// of the tile and ring formed), the load of the CTA's tile ST ahead is issued, so it runs under
// this tile's force, collision and observables.  One CTA barrier per tile: the psi / rho tile and
// the column sums are double-buffered by iteration parity, so a warp can start the next tile
// while others still read this one's.  Every wait on a load is bounded.
//
// Tiles are numbered in row-major order.  CTA b owns tiles b + i * grid for its first ST tiles
// (known before the previous kernel has finished, so its first load is issued as soon as that
// kernel's writes are visible); the rest are drawn from an atomic counter, one draw ahead, so the
// CTAs at work at any moment cover a band of rows and read each other's halo while it is in L2.
// A launch can also carry the reduction of the previous pass's observable partial sums (Fold):
// CTAs that have finished their tiles draw its work items from a second counter, so they fill the
// spread of the CTAs' last tiles; a CTA that looked at that counter during its last tile and saw
// no items left exits without drawing.  Launches alternate between two pairs of counters: each
// launch zeroes the pair the next launch will use, so no CTA has to find out that it is the last
// one out.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "lbm_pair.cuh"
#include "lbm_reduce.cuh"

namespace lbm {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int PZ = 8;   // tile rows
constexpr int BZ = PZ + 6;  // box rows: z0 - 3 .. z0 + PZ + 2 (padded z0 .. z0 + PZ + 5)
constexpr int HH = PZ + 4;  // psi/rho tile rows: z0 - 2 .. z0 + PZ + 1
// Tile shape: TW columns by PZ rows, one thread per site, TW = 32 (a warp per tile row) or 64 (two
// warps per tile row).  Row sums are formed per warp, over 32 columns, and column sums over the
// PZ rows, whatever the width: the partial sums, and so every result, do not depend on the shape.
template <int TW>
struct Shape {
    static constexpr int NT = TW * PZ;               // threads
    static constexpr int NW = NT / 32;               // warps
    static constexpr int BX = TW + 8;                // box columns: x0 - 4 .. x0 + TW + 3
    static constexpr int HW = TW + 4;                // psi/rho tile columns: x0 - 2 .. x0 + TW + 1
    static constexpr int NRING = HW * HH - TW * PZ;  // psi/rho tile positions outside the tile
    static constexpr int RPW = NRING / NW;           // ring positions per warp
    static_assert(NRING % NW == 0 && RPW <= 32, "the ring shared evenly over the warps");
    static_assert(NT % RB_THREADS == 0, "a CTA runs the reduction's work items");
};
// ST (template parameter): boxes in flight per CTA.  Width 32: 2, tiles loaded two ahead, 2 CTAs
// per SM in FP32; 1, one ahead, 3 CTAs per SM with fewer registers each.  Width 64: one CTA of 16
// warps per SM.  Chosen by lbm_autotune / lbm_autotune_tiles.
static_assert(PULL_GX == 4 && PULL_GZ == 3, "the box starts at padded (x0, z0)");

// Two species in FP32: the species go through the per-site arithmetic in lockstep (lbm_pair.cuh).
template <typename T, int NS>
constexpr bool kPair = sizeof(T) == 4 && NS == 2;

// psi and rho of the tile and its 2-cell ring: per species, or (species A, B) pairs
template <typename T, int NS, int TW, bool PAIR = kPair<T, NS>>
struct PsiTile {
    T ps[NS][HH][Shape<TW>::HW];
    T rh[NS][HH][Shape<TW>::HW];
};
template <int TW>
struct PsiTile<float, 2, TW, true> {
    f2 ps[HH][Shape<TW>::HW];
    f2 rh[HH][Shape<TW>::HW];
};

// Per-iteration ring of the tiles to work on: iteration k works on the tile described by
// ti[k % NTQ], published by thread 0 at the start of iteration k - ST (or before the loop), one
// CTA barrier ahead of every reader.
constexpr int NTQ = 4;

// A tile as thread 0 publishes it: its place and its lattice's geometry and drive, so that no
// other thread divides by the tile-row length or reads the lattice table.
template <typename T>
struct TileInfo {
    int t;          // tile number; >= the tile count: no more tiles
    int x0, z0;     // first column; first row among the rows of its lattice
    int jg;         // tile row among all lattices
    int lnz, zrow0; // its lattice's rows and first compact row
    int prow0;      // padded plane row of its lattice's row -PULL_GZ
    int pad_;
    T g, wall[2];   // its lattice's drive
};

template <typename T, int NS, int ST, int TW>
struct PullSmem {
    T box[ST][9 * NS][BZ][Shape<TW>::BX];  // TMA destinations (column bx = x - x0 + 4, row bz = z - z0 + 3)
    PsiTile<T, NS, TW> q[2];    // by iteration parity: tile k + 1 fills one while tile k reads the other
    T colsum[2][PZ][NQC][TW];   // by iteration parity: summed over the tile's rows one tile later
    typename Red<T>::A wsc[Shape<TW>::NW][NSC];  // folded reduction: per-warp scalars
    alignas(8) unsigned long long bar[ST];
    TileInfo<T> ti[NTQ];
    int fold_item;  // the reduction work item thread 0 drew for the CTA
    unsigned short ring[Shape<TW>::NT];  // observing builds: ring position of thread tid, rpz << 8 | rpx
};

// Tile t of the work order; rot > 0 (one periodic lattice): the order starts rot tiles in, at
// the last tile row, so the two rows whose sites also write the periodic row images come first
// and the last tiles of a launch are plain ones.  rev (one lattice, alternate launches): the tile
// rows in the opposite direction -- rows 0, ntz - 1, ntz - 2, ..., 1 when periodic (the image rows
// still first), ntz - 1 .. 0 between walls -- so that a launch starts on the rows the launch
// before wrote last, which may still be in L2.
template <typename T, int TW>
__device__ __forceinline__ void describe(TileInfo<T>& D, int t, int ntiles, const InstGeom* __restrict__ inst,
                                         int ninst, int ntx, int rot, int rev) {
    D.t = t;
    if (t >= ntiles) return;
    const InstGeom& I = inst[ninst > 1 ? inst_of_tile(inst, ninst, t / ntx) : 0];
    int tl = t - I.trow0 * ntx;
    if (rev && ninst == 1) {
        const int rp = tl / ntx, ntz = ntiles / ntx;
        const int row = rot > 0 ? (rp == 0 ? 0 : ntz - rp) : ntz - 1 - rp;
        tl = row * ntx + (tl - rp * ntx);
    } else if (rot > 0) {
        tl = tl < ntiles - rot ? tl + rot : tl - (ntiles - rot);
    }
    const int j = tl / ntx;
    D.x0 = (tl - j * ntx) * TW;
    D.z0 = j * PZ;
    D.jg = I.trow0 + j;
    D.lnz = I.nz;
    D.zrow0 = I.zrow0;
    D.prow0 = I.prow0;
    D.g = inst_g<T>(I);
    D.wall[0] = inst_wall_u<T>(I, 0);
    D.wall[1] = inst_wall_u<T>(I, 1);
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

template <typename T, int NS, int ST, int TW>
__device__ __forceinline__ void issue_load(PullSmem<T, NS, ST, TW>& S, const CUtensorMap* map, int x, int z, int sl) {
    constexpr unsigned bytes = (unsigned)(sizeof(T) * 9 * NS * BZ * Shape<TW>::BX);
    const unsigned bar = smem_u32(&S.bar[sl]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_u32(&S.box[sl][0][0][0])),
        "l"(map), "r"(x), "r"(z), "r"(0), "r"(bar)
        : "memory");
}

// Bounded wait for the phase of a load barrier: false once `limit` clock cycles have passed
// (the step kernel allows 2e9, about 1 s at 2 GHz).
constexpr long long WAIT_LIMIT = 2000000000LL;
__device__ __forceinline__ bool wait_load(unsigned bar, unsigned parity, long long limit = WAIT_LIMIT) {
    const long long t0 = clock64();
    for (;;) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

// Self-test of the bounded wait: one thread waits on a barrier that no copy and no thread ever
// completes, and records the expiry in flag bit 1 (as the step kernel does).
__global__ void k_wait_selftest(int* flag, long long limit) {
    __shared__ __align__(8) unsigned long long bar;
    const unsigned b = smem_u32(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(b) : "memory");
    if (!wait_load(b, 0u, limit)) atomicOr(flag, 2);
}

// Post-streaming populations at box position (bx, bz): the gather of the pull layout.  lo / hi:
// the site is the bottom / top row next to a wall, where populations coming from beyond the
// wall are the site's own reflected values.
template <typename T, int NS, int ST, int TW>
__device__ __forceinline__ void gather(const PullSmem<T, NS, ST, TW>& S, int sl, int bx, int bz, T (&f)[NS][9]) {
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int l = 0; l < 9; ++l) f[s][l] = S.box[sl][s * 9 + l][bz - cz(l)][bx - cx(l)];
}
template <typename T, int NS, int ST, int TW>
__device__ __forceinline__ void gather_wall(const PullSmem<T, NS, ST, TW>& S, int sl, int bx, int bz, bool lo, bool hi,
                                            T (&f)[NS][9]) {
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int l = 0; l < 9; ++l) {
            const bool refl = (cz(l) > 0 && lo) || (cz(l) < 0 && hi);
            f[s][l] = refl ? S.box[sl][s * 9 + opp(l)][bz][bx] : S.box[sl][s * 9 + l][bz - cz(l)][bx - cx(l)];
        }
}

// rho and psi at psi/rho tile position (px, pz) for a position that is not a live site of the
// tile: the ring, and the padding of ragged tiles.  With walls, rows beyond a wall take the
// mirror image (or zero, Sec. IV's two readings of the ghost rows).  Positions that no live
// site reads (far padding of ragged tiles) are set to zero.
template <typename T, int NS, int ST, int TW>
__device__ __forceinline__ void side_density(PullSmem<T, NS, ST, TW>& S, int sl, int qb, const StepConst<T>& C,
                                             const PairConst& K, int px, int pz, int z0, int nz, bool WALL) {
    const int Z = z0 - 2 + pz;
    int Zs = Z;
    bool zero = false;
    if (WALL && (Z < 0 || Z >= nz)) {
        if (C.psi_wall == 1)
            zero = true;
        else
            Zs = mirror_index(Z, nz);
    }
    const int bz = Zs - z0 + 3, bx = px + 2;
    if (bz < 1 || bz > BZ - 2) zero = true;
    T sum[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) sum[s] = T(0);
    if (!zero) {
        T g[NS][9];
        const bool lo = WALL && Zs == 0, hi = WALL && Zs == nz - 1;
        if (WALL && (lo || hi))
            gather_wall<T, NS, ST, TW>(S, sl, bx, bz, lo, hi, g);
        else
            gather<T, NS, ST, TW>(S, sl, bx, bz, g);
#pragma unroll
        for (int s = 0; s < NS; ++s) sum[s] = sum9(g[s]);
    }
    if constexpr (kPair<T, NS>) {
        const f2 rho = add2(K.rho_ref, p2(sum[0], sum[1]));
        S.q[qb].rh[pz][px] = zero ? sp(0.f) : rho;
        S.q[qb].ps[pz][px] = zero ? sp(0.f) : psi2(C, K, rho);
    } else {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const T rho = C.rho_ref[s] + sum[s];
            S.q[qb].rh[s][pz][px] = zero ? T(0) : rho;
            S.q[qb].ps[s][pz][px] = zero ? T(0) : psi_of(C, s, rho);
        }
    }
}

// The periodic images of site (x, z) of a lattice of nz rows whose row -PULL_GZ is padded row
// prow0: its new values, read back from where this thread has just stored them, copied into the
// ghost columns (and, without walls, ghost rows) that wrap onto it.
template <typename T, int NS>
__device__ __noinline__ void write_images(const StepConst<T>& C, T* __restrict__ fout, int x, int z, int nz,
                                          int prow0) {
    const int nx = C.nx;
    int xs[2 * PULL_GX + 1], zs[2 * PULL_GZ + 1];
    int nxs = 0, nzs = 0;
    xs[nxs++] = x;
    zs[nzs++] = z;
    for (int g = 0; g < 2 * PULL_GX; ++g) {
        const int gx = g < PULL_GX ? g - PULL_GX : nx + g - PULL_GX;
        if (wrap_index(gx, nx) == x) xs[nxs++] = gx;
    }
    if (!C.zbc)
        for (int g = 0; g < 2 * PULL_GZ; ++g) {
            const int gz = g < PULL_GZ ? g - PULL_GZ : nz + g - PULL_GZ;
            if (wrap_index(gz, nz) == z) zs[nzs++] = gz;
        }
    const T* src = fout + (long long)(prow0 + z + PULL_GZ) * C.pitch + (x + PULL_GX);
    T v[9 * NS];
#pragma unroll
    for (int p = 0; p < 9 * NS; ++p) v[p] = src[p * C.plane];
    for (int a = 0; a < nxs; ++a)
        for (int b = 0; b < nzs; ++b) {
            if (a == 0 && b == 0) continue;
            T* dst = fout + (long long)(prow0 + zs[b] + PULL_GZ) * C.pitch + (xs[a] + PULL_GX);
#pragma unroll
            for (int p = 0; p < 9 * NS; ++p) dst[p * C.plane] = v[p];
        }
}

// Ring position (psi/rho tile coordinates) of lane `lane` < RPW of warp `warp`: every warp has the
// same phase-A work (22 positions per warp at width 32, 19 at width 64); in ring order the top two
// rows, the bottom two rows, then two columns on each side of the tile rows.
template <int TW>
__device__ __forceinline__ void ring_position(int lane, int warp, int& rpx, int& rpz) {
    constexpr int HW = Shape<TW>::HW;
    const int k = warp * Shape<TW>::RPW + lane;
    if (k < 2 * HW) {
        rpz = k / HW;
        rpx = k % HW;
    } else if (k < 4 * HW) {
        rpz = HH - 2 + (k - 2 * HW) / HW;
        rpx = (k - 2 * HW) % HW;
    } else {
        const int j = k - 4 * HW;
        rpz = 2 + (j >> 2);
        const int c = j & 3;
        rpx = c < 2 ? c : HW - 4 + c;
    }
}

template <typename T, int NS, int MODE, int ST, int TW>
__global__ void __launch_bounds__(Shape<TW>::NT, TW == 64 ? 1 : (sizeof(T) == 4 ? (ST == 2 ? 2 : 3) : 1))
    k_pull(const __grid_constant__ CUtensorMap tin, T* __restrict__ fout,
           const StepConst<T> C, const PairConst K, const ObsPtrs O, const Fold Rd, unsigned* __restrict__ ctr,
           unsigned* __restrict__ ctr_next, const InstGeom* __restrict__ inst, int ninst, int ntx, int ntz,
           T* __restrict__ rec, int rev) {
    // walls in z: never in the periodic build, else as the step constants say
    const bool WALL = (MODE & M_PERIODIC) ? false : C.zbc != 0;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    using SH = Shape<TW>;
    PullSmem<T, NS, ST, TW>& S = *reinterpret_cast<PullSmem<T, NS, ST, TW>*>(smem_raw);
    const int tx = threadIdx.x, tz = threadIdx.y, tid = tz * TW + tx;
    const int nx = C.nx, nz = C.nz;
    const int ntiles = ntx * ntz;  // nz: rows of all lattices; ntz: their tile rows
    // tiles 0 .. nstat - 1 are owned by CTA (tile mod grid), the rest come from ctr[0]
    const int nstat = min(ST * (int)gridDim.x, ntiles);
    const int rot = !WALL && ninst == 1 && ntz > 2 ? ntiles - ntx : 0;  // work order (describe)
    // work items of the folded reduction: blocks of rows, then blocks of columns
    const int nrb = (nz + RB_THREADS / 32 - 1) / (RB_THREADS / 32);
    const int nfold = Rd.enabled ? nrb + (nx + RB_THREADS / 32 - 1) / (RB_THREADS / 32) : 0;

    // threads with a ring position (ring_position), RPW per warp; the observing builds keep it in
    // shared memory and read it per tile instead (one register pair less across the tile, where
    // registers are short), the others keep it in registers
    const bool ring = (tid & 31) < SH::RPW;
    int rpx0 = 0, rpz0 = 0;
    if (ring) ring_position<TW>(tid & 31, tid >> 5, rpx0, rpz0);
    if constexpr ((MODE & M_OBS) != 0) S.ring[tid] = (unsigned short)(rpz0 << 8 | rpx0);
    // thread 0 draws tiles one ahead of their loads, so the counter's latency is hidden;
    // ntiles: nothing more to draw
    int upcoming = ntiles;
    // the CTA's own first tiles, described before the previous kernel has finished: the lattice
    // table is written by host copies only, never by a kernel
    if (tid == 0) {
        for (int sl = 0; sl < ST; ++sl)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&S.bar[sl])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(&tin) : "memory");
        for (int sl = 0; sl < ST; ++sl) {
            const int t = (int)blockIdx.x + sl * (int)gridDim.x;
            if (t < nstat) describe<T, TW>(S.ti[sl], t, ntiles, inst, ninst, ntx, rot, rev);
        }
    }
    // Programmatic dependent launch: the next step's CTAs may be scheduled as soon as this grid's
    // CTAs start retiring; every thread of a grid waits for the previous grid's completion (and
    // the visibility of its writes) before its first access to the populations, the observable
    // buffers or the counters.
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    if (tid == 0) {
        if (blockIdx.x == 0) {  // the next launch's counters (this launch's were zeroed by the last)
            ctr_next[0] = 0u;
            ctr_next[1] = 0u;
        }
        // the first box goes out at once, the others once it has arrived (iteration 0), so that
        // the first boxes of all CTAs do not queue behind the second ones
        bool more = true;
        for (int sl = 0; sl < ST; ++sl) {
            if (!more) break;  // the slots after the CTA's first non-tile item stay unused
            const int t = (int)blockIdx.x + sl * (int)gridDim.x;
            if (t >= nstat)
                describe<T, TW>(S.ti[sl], min(nstat + (int)atomicAdd(ctr, 1u), ntiles), ntiles, inst, ninst, ntx,
                                rot, rev);
            more = S.ti[sl].t < ntiles;
            if (more && sl == 0) issue_load(S, &tin, S.ti[0].x0, S.ti[0].prow0 + S.ti[0].z0, 0);
        }
        if (more) upcoming = min(nstat + (int)atomicAdd(ctr, 1u), ntiles);
    }
    __syncthreads();
    // thread 0: the reduction's counter as last seen (no draw), during the CTA's last tiles
    int fold_seen = 0;
    unsigned parity = 0;  // bit sl: phase of box sl's barrier
    bool failed = false;
    // the previous tile's column-sum slot (observables): its column x and tile row, or x = -1
    int prev_x = -1, prev_jg = 0;
    int k = 0;
    for (;; ++k) {
        const int sl = k % ST, qb = k & 1;
        const TileInfo<T> D = S.ti[k % NTQ];
        if (D.t >= ntiles) break;
        if (tid == 0)  // publish the tile of iteration k + ST, one barrier ahead of its readers
            describe<T, TW>(S.ti[(k + ST) % NTQ], upcoming, ntiles, inst, ninst, ntx, rot, rev);
        // this tile: first column and row (rows of its lattice), tile row among all lattices; its
        // lattice: rows, first compact row, first padded row (the observing builds read them again
        // from shared memory after the tile barrier, so that they hold no registers across it)
        int lnz = D.lnz, zrow0 = D.zrow0, prow0 = D.prow0, x0 = D.x0, z0 = D.z0, jg = D.jg;
        int x = x0 + tx, z = z0 + tz;
        bool live = x < nx && z < lnz;
        const bool ok = wait_load(smem_u32(&S.bar[sl]), (parity >> sl) & 1u);
        if (ok) parity ^= 1u << sl;  // on expiry the exit path waits on the same phase again
        if (ST > 1 && k == 0 && tid == 0)  // the first box is in: the CTA's other first tiles
            for (int i = 1; i < ST; ++i) {
                if (S.ti[i].t >= ntiles) break;
                issue_load(S, &tin, S.ti[i].x0, S.ti[i].prow0 + S.ti[i].z0, i);
            }

        // ---- phase A: this site's populations, rho and psi of the tile and its ring ----
        T f[NS][9];
        T drho[NS];
        if (live) {
            const bool lo = WALL && z == 0, hi = WALL && z == lnz - 1;
            if (WALL && (lo || hi))
                gather_wall<T, NS, ST, TW>(S, sl, tx + 4, tz + 3, lo, hi, f);
            else
                gather<T, NS, ST, TW>(S, sl, tx + 4, tz + 3, f);
            if constexpr ((MODE & M_RECORD) != 0) {  // the input state, as plain values (one lattice)
                const long long n = (long long)nx * nz, i = (long long)z * nx + x;
#pragma unroll
                for (int s = 0; s < NS; ++s)
#pragma unroll
                    for (int l = 0; l < 9; ++l) rec[(s * 9 + l) * n + i] = f[s][l] + wlb<T>(l) * C.rho_ref[s];
            }
            if constexpr (kPair<T, NS>) {
                f2 fp[9];
#pragma unroll
                for (int l = 0; l < 9; ++l) fp[l] = p2(f[0][l], f[1][l]);
                const f2 d = sum9_2(fp);
                drho[0] = d.x;
                drho[NS - 1] = d.y;
                const f2 r = add2(K.rho_ref, d);
                S.q[qb].rh[tz + 2][tx + 2] = r;
                S.q[qb].ps[tz + 2][tx + 2] = psi2(C, K, r);
            } else {
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    drho[s] = sum9(f[s]);
                    const T r = C.rho_ref[s] + drho[s];
                    S.q[qb].rh[s][tz + 2][tx + 2] = r;
                    S.q[qb].ps[s][tz + 2][tx + 2] = psi_of(C, s, r);
                }
            }
        } else {
            side_density<T, NS, ST, TW>(S, sl, qb, C, K, tx + 2, tz + 2, z0, lnz, WALL);
        }
        if (ring) {
            int rpx = rpx0, rpz = rpz0;
            if constexpr ((MODE & M_OBS) != 0) {
                const unsigned rp = S.ring[tid];
                rpx = (int)(rp & 255u);
                rpz = (int)(rp >> 8);
            }
            side_density<T, NS, ST, TW>(S, sl, qb, C, K, rpx, rpz, z0, lnz, WALL);
        }
        // the only CTA barrier of a tile: psi / rho of the tile and ring complete, box sl read
        // by all, the previous tile's column sums written
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if constexpr ((MODE & M_OBS) != 0) {
            const TileInfo<T>& E = S.ti[k % NTQ];
            lnz = E.lnz;
            zrow0 = E.zrow0;
            prow0 = E.prow0;
            x0 = E.x0;
            z0 = E.z0;
            jg = E.jg;
            x = x0 + tx;
            z = z0 + tz;
            live = x < nx && z < lnz;
        }
        const int s = (x0 + (tx & ~31)) >> 5;  // this warp's group of 32 columns (row sums)
        // box sl is free: start the load of the tile ST ahead (published at the top of this
        // iteration) and draw the one after it; past the last tile, look at the reduction's
        // counter instead (its value is only used after the loop)
        if (tid == 0) {
            if (upcoming < ntiles) {
                const TileInfo<T>& N = S.ti[(k + ST) % NTQ];
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                issue_load(S, &tin, N.x0, N.prow0 + N.z0, sl);
                upcoming = min(nstat + (int)atomicAdd(ctr, 1u), ntiles);
            } else if (nfold > 0) {
                fold_seen = (int)*reinterpret_cast<volatile unsigned*>(ctr + 1);
            }
        }
        if (MODE & M_OBS) {
            // the previous tile's per-column sums over its PZ rows
            if (tz < NQC && prev_x >= 0 && prev_x < nx) {
                T v = T(0);
#pragma unroll
                for (int r = 0; r < PZ; ++r) v += S.colsum[qb ^ 1][r][tz][tx];
                static_cast<T*>(O.part_col)[((long long)prev_x * ntz + prev_jg) * NQC + tz] = v;
            }
            prev_x = x;
            prev_jg = jg;
        }

        // ---- phase B: interaction, collision, new stored values, observables ----
        const PsiTile<T, NS, TW>& Q = S.q[qb];
        T rowq[NQR];
#pragma unroll
        for (int q = 0; q < NQR; ++q) rowq[q] = T(0);
        T cps = T(0), cpx = T(0);
        int bad = 0;
        bool collided = false;  // f holds the post-collision values of a live site
        T rho[NS];
        if constexpr (kPair<T, NS>) {
            f2 Fx, Fz;
            float sxx = 0.f, szz = 0.f, sxz = 0.f;
            if constexpr ((MODE & M_OBS) != 0) {
                f2 a2, b2, c2;
                force_stress2<SH::HW>(K, &Q.ps[tz][tx], Fx, Fz, a2, b2, c2);
                sxx = a2.x + a2.y;
                szz = b2.x + b2.y;
                sxz = c2.x + c2.y;
            } else {
                f2 p[5][5];
#pragma unroll
                for (int dz = 0; dz < 5; ++dz)
#pragma unroll
                    for (int dx = 0; dx < 5; ++dx) p[dz][dx] = Q.ps[tz + dz][tx + dx];
                intra_force2(K, p, Fx, Fz);
            }
            f2 r[3][3];
#pragma unroll
            for (int dz = 0; dz < 3; ++dz)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) r[dz][dx] = Q.rh[tz + 1 + dz][tx + 1 + dx];
            cross_force2(K, r, Fx, Fz);
            if (MODE & M_OBS) cross_stress2(C, r, sxx, szz, sxz);
            if (live) {
                f2 fp[9];
#pragma unroll
                for (int l = 0; l < 9; ++l) fp[l] = p2(f[0][l], f[1][l]);
                const f2 dr = p2(drho[0], drho[1]);
                const f2 rh = add2(K.rho_ref, dr);
                rho[0] = rh.x;
                rho[1] = rh.y;
                if (!(rh.x > 0.f) || !(rh.x < 1e30f) || !(rh.y > 0.f) || !(rh.y < 1e30f)) bad = 1;
                const f2 ir = p2(__fdividef(1.f, rh.x), __fdividef(1.f, rh.y));
                f2 jx, jz;
                momentum9_2(fp, jx, jz);
                Fx = fma2(rh, sp(S.ti[k % NTQ].g), Fx);
                if (MODE & (M_OBS | M_FIELDS)) {
                    // barycentric velocity (sum_s j_s + F_s / 2) / sum_s rho_s and the kinetic flux
                    const f2 m = fma2(Fx, sp(0.5f), jx), n = fma2(Fz, sp(0.5f), jz);
                    const float mx = m.x + m.y, mz = n.x + n.y, rtot = rh.x + rh.y;
                    const float irt = __fdividef(1.f, rtot);
                    const float ux = mx * irt, uz = mz * irt;
                    if (MODE & M_FIELDS) {
                        const long long i = (long long)(zrow0 + z) * nx + x;
                        const long long np = (long long)nx * nz;
                        O.fields[i] = (double)rh.x;
                        O.fields[np + i] = (double)rh.y;
                        O.fields[2 * np + i] = (double)ux;
                        O.fields[3 * np + i] = (double)uz;
                    }
                    if (MODE & M_OBS) {
                        // xz second moment averaged over the collision (site_kinetics):
                        // (1 - omega/2) Pi + (omega/2) rho ueq_x ueq_z per species
                        const f2 pi = sub2(add2(fp[5], fp[7]), add2(fp[6], fp[8]));
                        const f2 wj = mul2(K.omega, jx), wk = mul2(K.omega, jz), wr = mul2(K.omega, rh);
                        const float iden = __fdividef(1.f, wr.x + wr.y);
                        const f2 tir = mul2(K.tau, ir);
                        const f2 ex = fma2(Fx, tir, sp((wj.x + wj.y) * iden));
                        const f2 ez = fma2(Fz, tir, sp((wk.x + wk.y) * iden));
                        const f2 v = fma2(K.half_om, pi, mul2(K.hom, mul2(rh, mul2(ex, ez))));
                        const float pixz = v.x + v.y;
                        const f2 third = mul2(rh, sp(1.f / 3.f));
                        const f2 kx2 = fma2(mul2(K.kin, mul2(Fx, Fx)), ir, third);
                        const f2 kz2 = fma2(mul2(K.kin, mul2(Fz, Fz)), ir, third);
                        const float pxx = sxx + (kx2.x + kx2.y), pzz = szz + (kz2.x + kz2.y);
                        cps = pxx - pzz;
                        cpx = pxx;
                        rowq[QR_UX] = ux;
                        rowq[QR_RHOA] = rh.x;
                        rowq[QR_RHOB] = rh.y;
                        rowq[QR_SXZ] = -pixz - sxz;
                        rowq[QR_MX] = mx;
                        rowq[QR_MZ] = mz;
                    }
                }
                const bool wall_row = WALL && (z == 0 || z == lnz - 1);
                if ((MODE & M_WRITE) || ((MODE & M_OBS) && wall_row)) {
                    collide2(K, fp, dr, rh, ir, jx, jz, Fx, Fz);
#pragma unroll
                    for (int l = 0; l < 9; ++l) {
                        f[0][l] = fp[l].x;
                        f[NS - 1][l] = fp[l].y;
                    }
                    collided = true;
                }
            }
        } else {
            T F[NS][2];
            T sxx = T(0), szz = T(0), sxz = T(0);
#pragma unroll
            for (int s2 = 0; s2 < NS; ++s2) {
                T p[5][5];
#pragma unroll
                for (int dz = 0; dz < 5; ++dz)
#pragma unroll
                    for (int dx = 0; dx < 5; ++dx) p[dz][dx] = Q.ps[s2][tz + dz][tx + dx];
                intra_force(C, s2, p, F[s2][0], F[s2][1]);
                if (MODE & M_OBS) intra_stress(C, s2, p, sxx, szz, sxz);
            }
            if constexpr (NS == 2) {
                T ra[3][3], rb[3][3];
#pragma unroll
                for (int dz = 0; dz < 3; ++dz)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
                        ra[dz][dx] = Q.rh[0][tz + 1 + dz][tx + 1 + dx];
                        rb[dz][dx] = Q.rh[1][tz + 1 + dz][tx + 1 + dx];
                    }
                cross_force(C, ra, rb, F);
                if (MODE & M_OBS) cross_stress(C, ra, rb, sxx, szz, sxz);
            }
            if (live) {
                T ir[NS], jx[NS], jz[NS];
#pragma unroll
                for (int s2 = 0; s2 < NS; ++s2) {
                    rho[s2] = C.rho_ref[s2] + drho[s2];
                    if (!(rho[s2] > T(0)) || !(rho[s2] < T(1e30))) bad = 1;
                    ir[s2] = div_(T(1), rho[s2]);
                    momentum9(f[s2], jx[s2], jz[s2]);
                    F[s2][0] += rho[s2] * S.ti[k % NTQ].g;
                }
                if (MODE & (M_OBS | M_FIELDS)) {
                    T ux, uz, pixz, rtot, mx, mz;
                    site_kinetics<T, NS>(C, f, rho, ir, jx, jz, F, ux, uz, pixz, rtot, mx, mz);
                    if (MODE & M_FIELDS) {
                        const long long i = (long long)(zrow0 + z) * nx + x;
                        const long long np = (long long)nx * nz;
#pragma unroll
                        for (int s2 = 0; s2 < NS; ++s2) O.fields[s2 * np + i] = (double)rho[s2];
                        O.fields[NS * np + i] = (double)ux;
                        O.fields[(NS + 1) * np + i] = (double)uz;
                    }
                    if (MODE & M_OBS) {
                        T pxx = sxx, pzz = szz;
#pragma unroll
                        for (int s2 = 0; s2 < NS; ++s2) {
                            pxx += rho[s2] * T(1.0 / 3.0) + C.kin[s2] * F[s2][0] * F[s2][0] * ir[s2];
                            pzz += rho[s2] * T(1.0 / 3.0) + C.kin[s2] * F[s2][1] * F[s2][1] * ir[s2];
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
                const bool wall_row = WALL && (z == 0 || z == lnz - 1);
                if ((MODE & M_WRITE) || ((MODE & M_OBS) && wall_row)) {
                    collide<T, NS>(C, f, drho, rho, ir, jx, jz, F);
                    collided = true;
                }
            }
        }
        // new stored values, straight from registers: a warp stores each plane's row of 32
        // sites as one 128-byte run; with walls the populations leaving through a wall reflected.
        // The periodic images of a site -- in the ghost columns when x is within PULL_GX of an
        // edge, and without walls in the ghost rows when z is within PULL_GZ of one -- take the
        // same values.  A lattice of at least 2 PULL_GX columns and 2 PULL_GZ rows gives a site at
        // most one image of each kind and their corner; they are stored here from registers, on
        // a branch that only warps holding such sites take.  Narrower lattices use write_images.
        T* const dst = fout + (long long)(prow0 + z + PULL_GZ) * C.pitch + (x + PULL_GX);
        const bool narrow = nx < 2 * PULL_GX || (!WALL && lnz < 2 * PULL_GZ);
        const int dxi = x < PULL_GX ? nx : (x >= nx - PULL_GX ? -nx : 0);
        const int dzi = WALL ? 0 : (z < PULL_GZ ? lnz : (z >= lnz - PULL_GZ ? -lnz : 0));
        const bool img = (MODE & M_WRITE) && collided && !narrow && (dxi != 0 || dzi != 0);
        const bool img_warp = __any_sync(FULL, img);  // every lane reaches this vote
        const long long oxi = dxi, ozi = (long long)dzi * C.pitch;
        if (collided) {
            const bool wall_row = WALL && (z == 0 || z == lnz - 1);
            if (!wall_row) {  // warp-uniform
                if (MODE & M_WRITE) {
                    if (img_warp) {
#pragma unroll
                        for (int s2 = 0; s2 < NS; ++s2)
#pragma unroll
                            for (int l = 0; l < 9; ++l) {
                                T* const p = dst + (s2 * 9 + l) * C.plane;
                                const T v = f[s2][l];
                                *p = v;
                                if (img) {
                                    if (dxi) p[oxi] = v;
                                    if (dzi) {
                                        p[ozi] = v;
                                        if (dxi) p[oxi + ozi] = v;
                                    }
                                }
                            }
                    } else {
#pragma unroll
                        for (int s2 = 0; s2 < NS; ++s2)
#pragma unroll
                            for (int l = 0; l < 9; ++l) dst[(s2 * 9 + l) * C.plane] = f[s2][l];
                    }
                }
            } else {
#pragma unroll
                for (int s2 = 0; s2 < NS; ++s2)
#pragma unroll
                    for (int l = 0; l < 9; ++l) {
                        const int zd = z + cz(l);
                        T v = f[s2][l];
                        if (zd < 0 || zd >= lnz) {  // leaves through a wall: store it reflected
                            const int w = zd < 0 ? 0 : 1;
                            const T back = bounce<T>(l, f[s2][l], rho[s2], S.ti[k % NTQ].wall[w]);
                            v = back;
                            if (MODE & M_OBS) {
                                const T dm = T(cx(l)) * (f[s2][l] + back);
                                if (w == 0)
                                    rowq[QR_WALLB] += dm;
                                else
                                    rowq[QR_WALLT] += dm;
                            }
                        }
                        if (MODE & M_WRITE) {
                            T* const p = dst + (s2 * 9 + l) * C.plane;
                            *p = v;
                            if (img && dxi) p[oxi] = v;  // walls: column images only
                        }
                    }
            }
        }
        if (__any_sync(FULL, bad) && tx == 0) atomicOr(O.flag, 1);
        if ((MODE & M_WRITE) && collided && narrow &&
            (x < PULL_GX || x >= nx - PULL_GX || (!WALL && (z < PULL_GZ || z >= lnz - PULL_GZ))))
            write_images<T, NS>(C, fout, x, z, lnz, prow0);
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
            if ((tx & 3) == 0 && z < lnz && (TW == 32 || (s << 5) < nx)) {  // a wide tile's warp may lie past nx
                const int q = (b4 ? 4 : 0) + (b3 ? 2 : 0) + (b2 ? 1 : 0);
                static_cast<T*>(O.part_row)[((long long)(zrow0 + z) * ((nx + 31) >> 5) + s) * NQR + q] = v1;
            }
            S.colsum[qb][tz][QC_PS][tx] = cps;
            S.colsum[qb][tz][QC_PXX][tx] = cpx;
        }
    }
    if ((MODE & M_OBS) && !failed) {
        // the last tile's per-column sums
        __syncthreads();
        if (tz < NQC && prev_x >= 0 && prev_x < nx) {
            T v = T(0);
#pragma unroll
            for (int r = 0; r < PZ; ++r) v += S.colsum[(k - 1) & 1][r][tz][tx];
            static_cast<T*>(O.part_col)[((long long)prev_x * ntz + prev_jg) * NQC + tz] = v;
        }
    }
    if (nfold > 0 && !failed) {
        // the previous pass's reduction: work items from the second counter until they run out
        for (;;) {
            if (tid == 0) S.fold_item = fold_seen < nfold ? (int)atomicAdd(ctr + 1, 1u) : nfold;
            __syncthreads();
            const int b = S.fold_item;
            if (b >= nfold) break;  // uniform: every thread read the same item
            reduce_block<T, (TW > 32)>(b, Rd.part_row, Rd.part_col, O.flag, Rd.nxpart, Rd.nzpart, nx, nz, C.zbc, nrb, Rd.out,
                            Rd.avg, Rd.bpart, Rd.bavg, Rd.accumulate, T(Rd.inx), T(Rd.inz), S.wsc,
                            ninst > 1 ? inst : nullptr, ninst);  // ends with a CTA barrier
        }
    }
    if (failed && tid == 0) {
        atomicOr(O.flag, 2);
        // the loads still in flight -- those of iterations k .. k + ST - 1 (the one that did not
        // arrive in time and the ones after it) -- before the CTA exits
        for (int i = 0; i < ST; ++i) {
            const int sl = (k + i) % ST;
            if (S.ti[(k + i) % NTQ].t < ntiles) wait_load(smem_u32(&S.bar[sl]), (parity >> sl) & 1u);
        }
    }
}

template <typename T, int NS, int MODE, int ST, int TW>
int pull_occupancy() {
    const size_t smem = sizeof(PullSmem<T, NS, ST, TW>);
    if (cudaFuncSetAttribute(k_pull<T, NS, MODE, ST, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_pull<T, NS, MODE, ST, TW>, Shape<TW>::NT, smem) !=
        cudaSuccess)
        return 0;
    return nb;
}

template <typename T, int NS, int MODE, int ST, int TW>
cudaError_t launch_mode(const void* tin, T* fout, const StepConst<T>& C, const ObsPtrs& O,
                        const Fold& Rd, unsigned* sched, int set, const Batch& B, int grid_max, cudaStream_t st,
                        T* rec) {
    const int ntx = (C.nx + TW - 1) / TW;
    const long long ntiles = (long long)ntx * B.ntz;
    int grid = (int)(ntiles < grid_max ? ntiles : grid_max);
    if (Rd.enabled && grid < 1) grid = 1;
    PairConst K{};
    if constexpr (kPair<T, NS>) fill_pair_const(K, C);
    // launched with programmatic stream serialisation: it may start while the kernel before it
    // on the stream drains, and waits for it in its prologue (griddepcontrol.wait)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(TW, PZ);
    cfg.dynamicSmemBytes = sizeof(PullSmem<T, NS, ST, TW>);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_pull<T, NS, MODE, ST, TW>, *static_cast<const CUtensorMap*>(tin), fout, C, K,
                              O, Rd, sched + 2 * set, sched + 2 * (set ^ 1), B.inst, B.ninst, ntx, B.ntz, rec,
                              set & 1);
}

// The passes built at width 64 as well: the FP32 step passes (lbm_step); all others run width 32.
template <typename T>
bool wide_pass(int mode) {
    return sizeof(T) == 4 && (mode == M_WRITE || mode == (M_WRITE | M_OBS) || mode == (M_PERIODIC | M_WRITE | M_OBS));
}

template <typename T, int NS, int ST, int TW>
cudaError_t launch_ns(int mode, const void* tin, T* fout, const StepConst<T>& C,
                      const ObsPtrs& O, const Fold& Rd, unsigned* sched, int set, const Batch& B, int grid_max,
                      cudaStream_t st, T* rec) {
#define LBM_PULL_CASE(m) \
    case m: return launch_mode<T, NS, m, ST, TW>(tin, fout, C, O, Rd, sched, set, B, grid_max, st, rec);
    if constexpr (TW == 32) {
        switch (mode) {
            LBM_PULL_CASE(M_WRITE)
            LBM_PULL_CASE(M_WRITE | M_OBS)
            LBM_PULL_CASE(M_OBS)
            LBM_PULL_CASE(M_FIELDS)
            LBM_PULL_CASE(M_PERIODIC | M_WRITE | M_OBS)
            LBM_PULL_CASE(M_PERIODIC | M_OBS)
            LBM_PULL_CASE(M_WRITE | M_RECORD)
            default: return cudaErrorInvalidValue;
        }
    } else if constexpr (sizeof(T) == 4) {
        switch (mode) {
            LBM_PULL_CASE(M_WRITE)
            LBM_PULL_CASE(M_WRITE | M_OBS)
            LBM_PULL_CASE(M_PERIODIC | M_WRITE | M_OBS)
            default: return cudaErrorInvalidValue;
        }
    } else {
        return cudaErrorInvalidValue;
    }
#undef LBM_PULL_CASE
}

// Ghost columns of every row of every lattice, and (one periodic lattice) the ghost rows, from
// the lattice values (after the initial state).
template <typename T>
__global__ void k_images(int ns, T* __restrict__ f, const StepConst<T> C, const InstGeom* __restrict__ inst,
                         int ninst) {
    const int wx = C.nx + 2 * PULL_GX;
    const long long nrow = (long long)C.nz * 2 * PULL_GX;          // x ghosts of the compact rows
    const long long nz_ghost = C.zbc ? 0 : (long long)2 * PULL_GZ * wx;  // ghost rows (single lattice)
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nrow + nz_ghost;
         i += (long long)gridDim.x * blockDim.x) {
        long long src, dst;
        if (i < nrow) {
            const int zg = (int)(i / (2 * PULL_GX)), g = (int)(i % (2 * PULL_GX));
            const int k = ninst > 1 ? inst_of_row(inst, ninst, zg) : 0;
            const int z = zg - inst[k].zrow0;
            const int gx = g < PULL_GX ? g - PULL_GX : C.nx + g - PULL_GX;
            const long long row = (long long)(inst[k].prow0 + z + PULL_GZ) * C.pitch;
            src = row + wrap_index(gx, C.nx) + PULL_GX;
            dst = row + gx + PULL_GX;
        } else {
            const long long q = i - nrow;
            const int gx = (int)(q % wx) - PULL_GX, r = (int)(q / wx);
            const int gz = r < PULL_GZ ? r - PULL_GZ : C.nz + r - PULL_GZ;
            src = (long long)(wrap_index(gz, C.nz) + PULL_GZ) * C.pitch + wrap_index(gx, C.nx) + PULL_GX;
            dst = (long long)(gz + PULL_GZ) * C.pitch + gx + PULL_GX;
        }
        for (int p = 0; p < 9 * ns; ++p) f[p * C.plane + dst] = f[p * C.plane + src];
    }
}

}  // namespace

template <typename T, int NS, int ST, int TW>
int blocks_per_sm_ns(int mode) {
#define LBM_PULL_CASE(m) \
    case m: return pull_occupancy<T, NS, m, ST, TW>();
    if constexpr (TW == 32) {
        switch (mode) {
            LBM_PULL_CASE(M_WRITE)
            LBM_PULL_CASE(M_WRITE | M_OBS)
            LBM_PULL_CASE(M_OBS)
            LBM_PULL_CASE(M_FIELDS)
            LBM_PULL_CASE(M_PERIODIC | M_WRITE | M_OBS)
            LBM_PULL_CASE(M_PERIODIC | M_OBS)
            LBM_PULL_CASE(M_WRITE | M_RECORD)
            default: return 0;
        }
    } else if constexpr (sizeof(T) == 4) {
        switch (mode) {
            LBM_PULL_CASE(M_WRITE)
            LBM_PULL_CASE(M_WRITE | M_OBS)
            LBM_PULL_CASE(M_PERIODIC | M_WRITE | M_OBS)
            default: return 0;
        }
    } else {
        return 0;
    }
#undef LBM_PULL_CASE
}

template <typename T, int ST, int TW>
int blocks_per_sm(int ns, int mode) {
    return ns == 1 ? blocks_per_sm_ns<T, 1, ST, TW>(mode) : blocks_per_sm_ns<T, 2, ST, TW>(mode);
}

template <typename T>
int pull_blocks_per_sm(int ns, int mode, int stages, int width) {
    if (width == 64) {
        if (!wide_pass<T>(mode)) return 0;
        return stages == 1 ? blocks_per_sm<T, 1, 64>(ns, mode) : blocks_per_sm<T, 2, 64>(ns, mode);
    }
    return stages == 1 ? blocks_per_sm<T, 1, 32>(ns, mode) : blocks_per_sm<T, 2, 32>(ns, mode);
}

template <typename T>
cudaError_t launch_pull(int ns, int mode, int stages, int width, const void* tin, T* fout,
                        const StepConst<T>& C, const ObsPtrs& O, const Fold& fold, unsigned* sched, int set,
                        const Batch& B, int grid_max, cudaStream_t st, T* rec) {
    if (set & ~1) return cudaErrorInvalidValue;
    if (grid_max < 1) return cudaErrorInvalidConfiguration;
    if (width == 64) {
        if (!wide_pass<T>(mode)) return cudaErrorInvalidValue;
        if (stages == 1)
            return ns == 1 ? launch_ns<T, 1, 1, 64>(mode, tin, fout, C, O, fold, sched, set, B, grid_max, st, rec)
                           : launch_ns<T, 2, 1, 64>(mode, tin, fout, C, O, fold, sched, set, B, grid_max, st, rec);
        return ns == 1 ? launch_ns<T, 1, 2, 64>(mode, tin, fout, C, O, fold, sched, set, B, grid_max, st, rec)
                       : launch_ns<T, 2, 2, 64>(mode, tin, fout, C, O, fold, sched, set, B, grid_max, st, rec);
    }
    if (stages == 1)
        return ns == 1 ? launch_ns<T, 1, 1, 32>(mode, tin, fout, C, O, fold, sched, set, B, grid_max, st, rec)
                       : launch_ns<T, 2, 1, 32>(mode, tin, fout, C, O, fold, sched, set, B, grid_max, st, rec);
    return ns == 1 ? launch_ns<T, 1, 2, 32>(mode, tin, fout, C, O, fold, sched, set, B, grid_max, st, rec)
                   : launch_ns<T, 2, 2, 32>(mode, tin, fout, C, O, fold, sched, set, B, grid_max, st, rec);
}

cudaError_t launch_wait_selftest(int* flag, long long cycles, cudaStream_t st) {
    k_wait_selftest<<<1, 1, 0, st>>>(flag, cycles);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pull_images(int ns, T* f, const StepConst<T>& C, const Batch& B, cudaStream_t st) {
    k_images<T><<<256, 256, 0, st>>>(ns, f, C, B.inst, B.ninst);
    return cudaGetLastError();
}

int make_pop_tmap(void* in_map, const void* f, int esize, int ns, int prows, int pitch, long long plane, int width) {
    const auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encoder());
    if (!encode) return 1;
    // the whole padded plane (prows rows), boxes of a tile and its 3-cell ring
    const cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)prows, (cuuint64_t)(9 * ns)};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * esize, (cuuint64_t)plane * esize};
    if (width != 32 && width != 64) return 3;
    const cuuint32_t box[3] = {(cuuint32_t)(width + 8), (cuuint32_t)BZ, (cuuint32_t)(9 * ns)};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt = esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    const CUresult r = encode(static_cast<CUtensorMap*>(in_map), dt, 3, const_cast<void*>(f), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : 2;
}

template int pull_blocks_per_sm<float>(int, int, int, int);
template int pull_blocks_per_sm<double>(int, int, int, int);
template cudaError_t launch_pull<float>(int, int, int, int, const void*, float*, const StepConst<float>&,
                                        const ObsPtrs&, const Fold&, unsigned*, int, const Batch&, int, cudaStream_t,
                                        float*);
template cudaError_t launch_pull<double>(int, int, int, int, const void*, double*, const StepConst<double>&,
                                         const ObsPtrs&, const Fold&, unsigned*, int, const Batch&, int, cudaStream_t,
                                         double*);
template cudaError_t launch_pull_images<float>(int, float*, const StepConst<float>&, const Batch&, cudaStream_t);
template cudaError_t launch_pull_images<double>(int, double*, const StepConst<double>&, const Batch&, cudaStream_t);

}  // namespace lbm
