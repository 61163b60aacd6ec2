// lbm_internal.h -- declarations shared by the library's translation units (not installed).
#pragma once

#include <cuda_runtime.h>

#include "lbm.h"
#include "lbm_core.cuh"

namespace lbm {

// Kernel modes (bit set).  M_PERIODIC (pull kernel only): compiled for periodic z, with no wall
// logic at all; without it the kernel reads the boundary from the step constants.  M_RECORD
// (pull kernel, with M_WRITE, one lattice): also writes the step's input state, the
// post-streaming populations as plain values, [ns][9][nz][nx] in the kernel's precision.
enum { M_WRITE = 1, M_OBS = 2, M_FIELDS = 4, M_PERIODIC = 8, M_RECORD = 16 };

// Width of the strip a warp owns in the fused sweep: 32 lanes minus a 2-column halo on
// each side (the reach of the 5x5 interaction stencil).
constexpr int STRIP_W = 28;

struct SweepGeom {
    int nstrips;  // ceil(nx / STRIP_W)
    int nchunks;  // ceil(nz / hz)
    int hz;       // rows swept by one warp
};

// Output pointers of the step kernels (device memory).  The partial sums are stored in the
// precision of the populations (float or double) and widened to FP64 by the reduction.
struct ObsPtrs {
    void* part_row;    // [nz][nxpart][NQR]   per-row sums over a group of columns
    void* part_col;    // [nx][nzpart][NQC]   per-column sums over a group of rows
    double* fields;    // [ns + 2][nz][nx]    rho_s, u_x, u_z (M_FIELDS)
    int* flag;         // bit 0: a density <= 0 / NaN / Inf was met
};

// Two-pass layout: densities and pseudopotentials with ghost cells (2 rows above and
// below, GX columns left and right), pitch gpitch elements, one plane per field.
constexpr int GX = 4;
struct GhostGeom {
    int gpitch;           // >= nx + 2 GX, multiple of 4 (16-byte rows for TMA)
    long long gplane;     // (nz + 4) * gpitch
};

// Observable output layout (doubles) written by the reduction kernel: scalars, then the row
// profiles ux_z, rho_z[2], sxz_z, fluid_z, the column profiles ps_x, pxx_x, and the row profiles
// mx_z, mz_z (x-averaged momentum) and wallb_z, wallt_z (x-averaged wall momentum exchange,
// nonzero on a lattice's first / last row).  nz counts all rows of a stacked batch.
enum { O_MASS = 0, O_MOM = 2, O_GAMMA = 4, O_WALL = 5, O_BAD = 7, O_COUNT = 8, O_PROF = 16 };
LBM_HD long long obs_len(int nx, int nz) { return O_PROF + 9LL * nz + 2LL * nx; }

// One lattice of a stacked batch (a single lattice is a batch of one).  All lattices share nx
// and the model parameters except the drive; lattice i's rows follow lattice i - 1's, in the
// fields' layout (compact rows) and in the population planes (each with its own ghost rows).
struct InstGeom {
    int nz;       // rows of the lattice
    int zrow0;    // its row 0 among the compact rows of the batch
    int prow0;    // padded plane row of its row -PULL_GZ (its row z sits at prow0 + PULL_GZ + z)
    int trow0;    // its first tile row in the pull kernel's numbering (tiles of PZ = 8 rows)
    int ntz;      // its tile rows
    float g_f;           // g in FP32 (set with g: the FP32 kernels issue no FP64 conversion)
    double g;            // body acceleration along x
    double wall_u[2];    // bottom, top wall velocity along x
    float wall_u_f[2];   // wall_u in FP32
    int pad2_[2];
};
// The drive of a lattice in the kernels' precision.
template <typename T>
LBM_HD T inst_g(const InstGeom& I) {
    if constexpr (sizeof(T) == 4) return I.g_f; else return I.g;
}
template <typename T>
LBM_HD T inst_wall_u(const InstGeom& I, int w) {
    if constexpr (sizeof(T) == 4) return I.wall_u_f[w]; else return I.wall_u[w];
}
// Sets a lattice's drive (both precisions).
// The densities of lbm_set_fields checked and summed on the device.  rho [ns][n] (device memory);
// scratch: DCHECK_DOUBLES doubles of device memory.  The kernels leave in scratch: [0], [1] the
// sums over each species' n values (a fixed order, the same bits on every call); [2], as an
// unsigned 64-bit integer, the first index s n + i of a value that is not > 0 and finite, or all
// ones.  Enqueued on st; the caller reads the three values back.
constexpr int DCHECK_BLOCKS = 256;
constexpr int DCHECK_DOUBLES = 3 + 2 * DCHECK_BLOCKS;
cudaError_t launch_density_check(const double* rho, long long n, int ns, double* scratch, cudaStream_t st);

inline void set_inst_drive(InstGeom& I, double g, double wb, double wt) {
    I.g = g;
    I.g_f = (float)g;
    I.wall_u[0] = wb;
    I.wall_u[1] = wt;
    I.wall_u_f[0] = (float)wb;
    I.wall_u_f[1] = (float)wt;
}
// The lattices of a pull-kernel context, as the kernels see them: the device copy of the table,
// its length, and the tile rows of all lattices together.
struct Batch {
    const InstGeom* inst;
    int ninst;
    int ntz;
};

// The lattice holding compact row zg, or tile row tr (binary search over ascending starts).
LBM_HD int inst_of_row(const InstGeom* I, int n, int zg) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (I[mid].zrow0 <= zg)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}
LBM_HD int inst_of_tile(const InstGeom* I, int n, int tr) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (I[mid].trow0 <= tr)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Launchers (return the launch error).
template <typename T>
cudaError_t launch_fused(int ns, int mode, const T* fin, T* fout, const StepConst<T>& C, const SweepGeom& G,
                         const ObsPtrs& O, cudaStream_t st);
// One-pass tile kernel; tile_rows = 8 or 16 (tile height).
template <typename T>
cudaError_t launch_tile(int ns, int mode, int tile_rows, const T* fin, T* fout, const StepConst<T>& C,
                        const ObsPtrs& O, cudaStream_t st);
// Warps of the sweep kernel resident on the whole GPU at once (occupancy), for a mode class.
template <typename T>
int fused_resident_warps(int ns, int mode, int nsm);
template <typename T>
cudaError_t launch_density(int ns, const T* f, T* gfield, const StepConst<T>& C, const GhostGeom& GG,
                           cudaStream_t st);
template <typename T>
cudaError_t launch_twopass(int ns, int mode, const T* fin, T* fout, const T* gfield, const StepConst<T>& C,
                           const GhostGeom& GG, const void* tmap, const ObsPtrs& O, int nxpart, int nzpart,
                           cudaStream_t st);
// The CUDA driver API's cuTensorMapEncodeTiled (resolved once through the runtime), or null.
void* tensor_map_encoder();
// Encodes the TMA descriptor (CUtensorMap, 128 bytes at out) of the two-pass field planes.
// Returns 0 on success.
int make_field_tmap(void* out, const void* g, int esize, int ns, int nz, const GhostGeom& GG);
// The reduction of an earlier pass's partial sums, folded into a pull-kernel launch (its CTAs
// run the work items of the reduction kernel before their first tile).  Pointers as for
// launch_reduce; enabled = 0: nothing to reduce.
struct Fold {
    const void* part_row;
    const void* part_col;
    double* out;
    double* avg;
    double* bpart;
    double* bavg;
    int nxpart, nzpart;
    int accumulate;
    int enabled;
    double inx, inz;  // 1/nx, 1/nz
};

// Pull layout: ghost columns on either side and ghost rows above and below each lattice in the
// plane; lattice site (x, z) sits at padded column x + PULL_GX, padded row prow0 + z + PULL_GZ
// (prow0 = 0 for a single lattice).  pitch >= nx + 2 PULL_GX, plane = prows * pitch with
// prows = sum over the lattices of (nz + 2 PULL_GZ).
constexpr int PULL_GX = 4, PULL_GZ = 3;

// Pull-layout kernel: the TMA descriptor (CUtensorMap, 128 bytes at in_map) of one population
// buffer f ([9 ns][prows][pitch] values) for loading the box of a tile of `width` (32 or 64)
// columns and its 3-cell ring.  Returns 0 on success.
int make_pop_tmap(void* in_map, const void* f, int esize, int ns, int prows, int pitch, long long plane,
                  int width);
// CTAs of the pull kernel resident per SM for a mode, a pipeline depth (stages = boxes in flight
// per CTA, 1 or 2) and a tile width (32, or 64 for the FP32 step passes M_WRITE, M_WRITE | M_OBS,
// M_PERIODIC | M_WRITE | M_OBS); sets the kernel's shared-memory limit on the current device; 0
// on failure or for a width the mode is not built at.
template <typename T>
int pull_blocks_per_sm(int ns, int mode, int stages, int width);
// One pass of the pull kernel: loads through tin (a buffer's in_map) and stores the new values
// into fout, the other buffer (their periodic images too).  fold: a pending reduction run by the same launch.  sched: two
// pairs of work-item counters (tiles, reduction items); consecutive launches of a context
// alternate set = 0, 1, 0, ...: a launch uses pair `set`, which must be zero when it starts, and
// zeroes the other pair for the next.
// grid_max: resident CTAs on the device.
template <typename T>
cudaError_t launch_pull(int ns, int mode, int stages, int width, const void* tin, T* fout,
                        const StepConst<T>& C, const ObsPtrs& O, const Fold& fold, unsigned* sched, int set,
                        const Batch& B, int grid_max, cudaStream_t st, T* rec = nullptr);
// One thread waits `cycles` clock cycles on a barrier nothing completes, then sets bit 1 of *flag.
cudaError_t launch_wait_selftest(int* flag, long long cycles, cudaStream_t st);
// Fills the ghost columns and rows of a pull-layout buffer with the periodic images.
template <typename T>
cudaError_t launch_pull_images(int ns, T* f, const StepConst<T>& C, const Batch& B, cudaStream_t st);
// Initial state / export of the populations of Sec. II (post-streaming, plain FP64 values),
// in the push layout (B null) or the padded pull layout of the pull kernel's lattices (C.pitch,
// C.plane are the buffer's; the ghosts are filled by launch_pull_images).
template <typename T>
cudaError_t launch_init(int ns, T* f, const double* rho, const double* u, const StepConst<T>& C, const Batch* B,
                        cudaStream_t st);
template <typename T, typename O>
cudaError_t launch_export(int ns, const T* f, O* out, const StepConst<T>& C, const Batch* B, cudaStream_t st);
// The inverse of launch_export: plain FP64 post-streaming populations in, the stored layout out
// (deviations from W_l rho_ref); the pull layout's ghosts are filled by launch_pull_images.
template <typename T>
cudaError_t launch_import(int ns, T* f, const double* in, const StepConst<T>& C, const Batch* B, cudaStream_t st);
// Reduction of the step kernels' partial sums into the observables.  `out` / `avg` hold
// obs_len(nx, nz) entries (profiles, wall forces, flag); `bpart` / `bavg` hold
// reduce_blocks(nx, nz) * 5 block partials of the scalars (mass A, B, momentum x, z, gamma) and
// their time sums.  With tail the scalar sums are also written into out[O_MASS..].  Entries are
// doubles (FP64 mode) or (hi, lo) float pairs (FP32 mode).  inst / ninst: the device table of a
// stacked batch (rows of different lattices are not neighbours), null for one lattice.
int reduce_blocks(int nx, int nz);
// Writes the trailer of an asynchronous read (samples, step, averages, 0: four 8-byte words) at
// dst, in device memory, in stream order.
cudaError_t launch_obs_trailer(double* dst, double samples, long long step, long long averages, cudaStream_t st);
// Sets bit 4 of *flag when the 8-byte tag at `tag` is not `expected` (a snapshot restored from
// the host's record of it had been overwritten since).
cudaError_t launch_snap_check(const unsigned long long* tag, unsigned long long expected, int* flag,
                              cudaStream_t st);
cudaError_t launch_reduce(int precision_bytes, const ObsPtrs& O, int nxpart, int nzpart, int nx, int nz, int zbc,
                          unsigned* ticket, double* out, double* avg, double* bpart, double* bavg, int accumulate,
                          bool tail, const InstGeom* inst, int ninst, cudaStream_t st);

// Discrete adjoint of the step on a periodic lattice (FP64, plain [ns][9][nz][nx] layouts).
// Couplings and weights as the step uses them: wa / wr / wc = weight_norm x the attraction,
// repulsion and cross weights by |c|^2.
struct AdjConst {
    int nx, nz, ns, psi_form;
    double wa[9], wr[9], wc[9];
    double G1[2], G2[2], tau[2], rho0[2];
    double G_AB, g;
};
void fill_adj_const(AdjConst& A, const lbm_params& p, int nx, int nz, int ns, double body_force);
// Bytes of scratch the adjoint launches need (one buffer serves all of them, used in turn).
size_t adjoint_scratch_bytes(int nx, int nz, int ns);
// nsteps adjoint steps backwards over the states f_k .. f_{k+nsteps-1} (states[j] at
// states + j stride): lam_in = dJ/df_{k+nsteps}; the steps write alternately into lam_a and
// lam_b (neither may be lam_in's buffer while it is read: lam_b may be it, it is first written
// by the second step); *lam_out receives the buffer holding dJ/df_k (lam_in when nsteps = 0).
// Adds dJ/dtheta to grad[8].  T = double or float.  ev: null, or 6 events per step recorded
// around its three kernels (before / after each, in launch order).
template <typename T>
cudaError_t launch_adjoint_steps(const AdjConst& D, int nsteps, const T* states, long long stride, const T* lam_in,
                                 T* lam_a, T* lam_b, const T** lam_out, double* grad, void* scratch, cudaEvent_t* ev,
                                 cudaStream_t st);
// J (one double) of the velocity / density profile objective at f and, when g is not null,
// g = dJ/df.
template <typename T>
cudaError_t launch_adjoint_objective(const AdjConst& D, const T* f, const double* tu, const double* tr, double* J,
                                     T* g, void* scratch, cudaStream_t st);
// g [ns][nz][nx] = sum_l W_l lam0: the derivative with respect to the densities of an initial
// state at rest.
template <typename T>
cudaError_t launch_adjoint_initial(const AdjConst& D, const T* lam0, double* g, cudaStream_t st);

// Twopass tile (threads per CTA: TPX x TPZ sites).
constexpr int TPX = 32, TPZ = 8;

}  // namespace lbm
