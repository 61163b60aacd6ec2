/*
 * lbm.h -- C ABI of liblbm.so, the GB300 (sm_103a) implementation of the time step of the
 * two-belt ("frustrated") multirange Shan-Chen lattice Boltzmann model for non-ideal fluids
 * and A/B emulsions of Sbragaglia, Benzi, Bernaschi and Succi, "The emergence of
 * supramolecular forces from lattice kinetic models of non ideal fluids: applications to the
 * rheology of soft glassy materials" (arXiv:1402.6019).
 *
 * Conventions for every call:
 *  - Return value: LBM_OK (0) or a positive LBM_E* code.  No call throws and no call aborts
 *    the process.  lbm_last_error() gives a one-line description of the last failure on
 *    that context.
 *  - Lattice: x (stream-flow, periodic) is the fastest index, z (cross-flow) the slower one,
 *    as in Sec. IV.  Host arrays are C-contiguous FP64 in the layouts stated per call.
 *  - Memory: host arrays passed in are copied before the call returns; host arrays passed
 *    out are written before it returns.  "where" = LBM_DEVICE means the pointer is CUDA
 *    device memory on the context's device, read or written on the context's stream and
 *    owned by the caller.  The library owns all device memory it allocates and frees it in
 *    lbm_destroy.
 *  - Streams: calls that launch work enqueue it on the context's stream and return without
 *    waiting, except where a call says it synchronises.
 *  - A context is bound to one device and one stream and is not thread-safe.
 */
#ifndef LBM_H
#define LBM_H

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_ABI_VERSION 5

/* status codes */
enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,     /* bad argument; nothing was changed                          */
    LBM_ECUDA = 2,      /* a CUDA call failed (no device, launch error, ...)           */
    LBM_ENOMEM = 3,     /* device or host allocation failed                            */
    LBM_ENONFINITE = 4, /* the state holds a density that is <= 0, NaN or Inf           */
    LBM_ETIMEOUT = 5    /* a bounded device-side wait gave up                          */
};

enum { LBM_FP64 = 0, LBM_FP32 = 1 };            /* storage + arithmetic of the populations  */
enum { LBM_PERIODIC = 0, LBM_BOUNCEBACK = 1 };  /* boundary in z (x is always periodic)     */
/* step kernels: PULL = one pass of persistent CTAs on 2-D tiles moved by TMA tensor loads and
   stores, populations kept in the pull layout (post-collision values; the default, AUTO);
   FUSED = one pass on 2-D tiles with the density halo recomputed from plain loads;
   TWO_PASS = a density/psi pass, then a collide pass staging the psi/rho tile by TMA;
   SWEEP = one pass of warp strips sweeping rows with a cp.async shared-memory ring.
   FUSED, TWO_PASS and SWEEP keep the push layout (post-streaming values).  The layout is
   internal: every entry point takes and returns the post-streaming populations of Sec. II. */
enum { LBM_KERNEL_AUTO = 0, LBM_KERNEL_FUSED = 1, LBM_KERNEL_TWO_PASS = 2, LBM_KERNEL_SWEEP = 3, LBM_KERNEL_PULL = 4 };
enum { LBM_PSI_EXP = 0, LBM_PSI_RHO = 1 };
enum { LBM_WEIGHTS_PAPER = 0, LBM_WEIGHTS_CHEM09 = 1 };
enum { LBM_WALL_MIRROR = 0, LBM_WALL_ZERO = 1 };
enum { LBM_HOST = 0, LBM_DEVICE = 1 };

typedef struct lbm_ctx lbm_ctx;

/* Lattice and execution description, fixed for the life of a context. */
typedef struct {
    int nx, nz;          /* lattice size, 1 <= nx, nz <= 65536, nx * nz <= 2^30          */
    int n_species;       /* 1 (Secs. II-III) or 2 (the A/B emulsion of Sec. IV)          */
    int precision;       /* LBM_FP64, or LBM_FP32: populations stored and relaxed in FP32
                            as deviations f_l - W_l rho_ref from the rest weights           */
    int z_boundary;      /* LBM_PERIODIC or LBM_BOUNCEBACK (walls at z = -1/2, nz - 1/2)  */
    int kernel;          /* LBM_KERNEL_AUTO / _PULL / _FUSED / _TWO_PASS / _SWEEP (above)   */
    int device;          /* CUDA device ordinal                                          */
    void *stream;        /* cudaStream_t to run on; NULL = a stream owned by the context  */
    int rows_per_warp;   /* SWEEP kernel: rows of one strip swept by a warp; 0 = auto      */
    int tile_rows;       /* FUSED kernel: tile height, 8 or 16 rows; 0 = auto             */
    int n_instances;     /* 0 or 1: one lattice.  > 1: a batch of that many channels (at
                            most 4096) stepped together by the PULL kernel: lattice i has
                            inst_nz[i] rows, the same nx, couplings and walls
                            (LBM_BOUNCEBACK), its own drive (lbm_set_instance_drive), and
                            nz must equal the sum of inst_nz.  Fields and profiles of the
                            batch stack the lattices' rows in order.                      */
    const int *inst_nz;  /* n_instances > 1: host array of the lattices' heights (read by
                            lbm_create only)                                              */
} lbm_desc;

/* Model parameters (Eq. LB, Eq. FORCE, Sec. IV).  Species index 0 = A, 1 = B. */
typedef struct {
    double tau[2];       /* BGK relaxation time (Eq. LB), > 1/2                          */
    double G1[2];        /* short-range (attractive, < 0) coupling of Eq. FORCE            */
    double G2[2];        /* mid-range (repulsive, > 0) coupling of Eq. FORCE               */
    double G_AB;         /* A-B cross repulsion of Sec. IV                                */
    int psi_form;        /* LBM_PSI_EXP: psi = 1 - exp(-rho/rho0) (Sec. IV); LBM_PSI_RHO  */
    double rho0[2];      /* rho0 of the exponential pseudopotential, > 0                  */
    int weight_preset;   /* LBM_WEIGHTS_PAPER: attraction on |c|^2 <= 4 (l = 1..12),
                            repulsion on |c|^2 <= 8 (l = 1..24), both 6th-order isotropic
                            (Eq. FORCE); LBM_WEIGHTS_CHEM09: attraction on the first belt    */
    double weight_norm;  /* scale of every interaction weight: the tables of Appendix B
                            have sum W c c = 1; Eq. BULK corresponds to 1/3               */
    double body_force;   /* acceleration g along x: F_s += rho_s g (Sec. IV drive)        */
    double wall_u[2];    /* x-velocity of the bottom and top walls (Sec. IV Couette)      */
    int psi_wall;        /* psi and rho in the two ghost rows beyond a wall: mirror image
                            of the fluid (LBM_WALL_MIRROR) or zero (LBM_WALL_ZERO)          */
    double rho_ref[2];   /* LBM_FP32 only: reference density of the stored deviations;
                            < 0 selects the mean density given to lbm_set_fields            */
} lbm_params;

/* Observables of one state (Secs. III-IV), FP64.  Profile pointers are caller-owned host
   arrays or NULL to skip. */
typedef struct {
    double mass[2];        /* sum over sites of rho_s                                      */
    double momentum[2];    /* sum over sites and species of j_s + F_s / 2                  */
    double gamma;          /* sum over x of the z-average of P_xx - P_zz (Eq. DIS1): the
                              surface tension of interfaces normal to x                     */
    double wall_force[2];  /* x-momentum given per step and unit length to the bottom and
                              top wall by bounce-back (zero without walls)                  */
    int nonfinite;         /* 1 if a density <= 0, NaN or Inf was met                      */
    long long step;        /* steps taken since lbm_set_fields                             */
    long long samples;     /* lbm_averages: number of states averaged                      */
    double *ux_z;          /* [nz] x-average of the barycentric velocity u_x               */
    double *rho_z;         /* [n_species][nz] x-average of rho_s                          */
    double *sxz_z;         /* [nz] x-average of the shear stress S_xz                      */
    double *fluid_z;       /* [nz] fluidity (d ux_z / dz) / sxz_z (Eq. fluidity)            */
    double *ps_x;          /* [nx] z-average of P_xx - P_zz                                */
    double *pxx_x;         /* [nx] z-average of the normal pressure P_xx (Sec. III)        */
} lbm_obs;

/* Create a context: validates d, selects d->device, allocates the double-buffered
   populations and the reduction buffers.  *out is NULL on failure. */
int lbm_create(lbm_ctx **out, const lbm_desc *d);

/* Check a description without touching any GPU (LBM_OK or LBM_EINVAL). */
int lbm_validate_desc(const lbm_desc *d);
/* Check parameters for a context with n_species species without touching any GPU. */
int lbm_validate_params(const lbm_params *p, int n_species);
/* Fill d and p with the defaults (1 species, FP64, periodic; tau = 1, weight_norm = 1/3). */
void lbm_default_desc(lbm_desc *d);
void lbm_default_params(lbm_params *p);

/* Set the model parameters (Eq. LB tau, Eq. FORCE G1/G2 and weights, Sec. IV G_AB, psi
   form, drives).  Takes effect from the next step. */
int lbm_set_params(lbm_ctx *c, const lbm_params *p);

/* Initial state: populations at the equilibrium of Sec. II for the given densities
   rho [n_species][nz][nx] (every value > 0 and finite) and velocity u [2][nz][nx] (NULL:
   u = 0).  Resets the step counter and the time averages.  Synchronises the stream. */
int lbm_set_fields(lbm_ctx *c, const double *rho, const double *u, int where);

/* Read the state.  Any pointer may be NULL.  rho [n_species][nz][nx]; u [2][nz][nx], the
   barycentric velocity (sum_s j_s + F_s/2) / sum_s rho_s; f [n_species][9][nz][nx], the
   populations after streaming (FP64; FP32 deviations are converted).  Synchronises. */
int lbm_get_fields(lbm_ctx *c, double *rho, double *u, double *f, int where);

/* Advance nsteps >= 0 time steps (Eq. LB with the force of Eq. FORCE applied by the shifted
   velocity of Sec. II, then streaming with the walls of Sec. IV).  Asynchronous.  While
   sampling is on (lbm_set_observe), every k-th step also accumulates the observables of
   the state it collides into FP64 time sums on the device.
   Captured into a caller's CUDA graph (stream capture on the context's stream), the launches
   are recorded with their arguments and the context's host-side state advances as if they had
   run: the step counter, the pending observables pass, and the pair of work counters that
   consecutive launches alternate.  Replay such a graph once per capture.  A second replay
   would start from a state the context has moved past (with an odd number of steps captured,
   its first launch would also find a work counter it expects to be zero still holding the last
   count). */
int lbm_step(lbm_ctx *c, int nsteps);

/* Sampling of time averages: every k >= 1 steps, or 0 = off.  Resets the sums. */
int lbm_set_observe(lbm_ctx *c, int every);

/* Observables of the current state.  Synchronises the stream. */
int lbm_observables(lbm_ctx *c, lbm_obs *out);

/* Time averages of the observables sampled since the last reset (out->samples of them);
   reset != 0 clears the sums afterwards.  Synchronises the stream. */
int lbm_averages(lbm_ctx *c, lbm_obs *out, int reset);

/* Reading observables without waiting (no counterpart in the paper): lets a caller overlap the
   read-back of one step's observables with the next step.
   lbm_observables_enqueue enqueues on the context's stream what lbm_observables (averages = 0)
   or lbm_averages (averages = 1; reset != 0 clears the sums after the copy) compute, copying
   the raw record -- lbm_observables_bytes(c) bytes -- into dst (pinned host memory, or device
   memory), and returns without waiting; *ticket (may be NULL) identifies the enqueue.
   averages = 2: the time sums as they stand, without the reduction of the last observing step
   if it is still pending (the next step's launch adds it; it is counted in the next record), so
   no separate reduction is launched -- when every step samples, each record then holds the
   step before the last.
   lbm_wait waits until the work enqueued up to that ticket is done (an event; the last 64
   tickets are tracked, older ones wait for the whole stream).  lbm_observables_unpack turns a
   record that has arrived into lbm_obs (host arithmetic only; returns LBM_ENONFINITE for a
   current-state record whose state held a bad density). */
long long lbm_observables_bytes(const lbm_ctx *c);
int lbm_observables_enqueue(lbm_ctx *c, void *dst, int averages, int reset, long long *ticket);
int lbm_wait(lbm_ctx *c, long long ticket);
int lbm_observables_unpack(const lbm_ctx *c, const void *src, lbm_obs *out);

/* A time series of observables in one call (no counterpart in the paper): nsteps (>= 0) times,
   one step (lbm_step(c, 1)) followed by lbm_observables_enqueue(c, dst + i * stride, averages,
   reset), so the host spends one call, not two per step, and the records go out while the
   next steps run.  stride >= lbm_observables_bytes(c); dst must hold nsteps records (pinned host
   or device memory; the caller owns it and keeps it until the records have arrived).  *ticket
   (may be NULL) receives the ticket of the last record (lbm_wait on it waits for all of them).
   Stops at the first error and returns it; the steps and records before it stay enqueued. */
int lbm_step_read(lbm_ctx *c, int nsteps, void *dst, long long stride, int averages, int reset,
                  long long *ticket);

/* Wait for the context's stream; reports LBM_ENONFINITE if a step met a bad density. */
int lbm_synchronize(lbm_ctx *c);

/* Number of kernels the context has launched so far (all kinds). */
long long lbm_launch_count(const lbm_ctx *c);

/* Kernel timing: while enabled (enable != 0), every launch of the step kernel made by
   lbm_step is bracketed by CUDA events on the context's stream (CUDA-graph replay is off),
   and lbm_profile_read returns the summed event time in milliseconds and the number of
   launches timed since profiling was enabled.  lbm_profile_read synchronises. */
int lbm_profile(lbm_ctx *c, int enable);
int lbm_profile_read(lbm_ctx *c, double *step_kernel_ms, long long *launches);
/* While profiling is enabled, every adjoint step (lbm_adjoint_step, lbm_adjoint_steps) also
   brackets each of its three kernels with CUDA events: ms[3] receives their summed times in
   milliseconds (moments, local, final) and steps the adjoint steps timed.  Synchronises. */
int lbm_profile_read_adjoint(lbm_ctx *c, double *ms, long long *steps);

/* One-line description of the last failure on c (or of the last lbm_create failure when
   c is NULL).  Valid until the next call on c. */
const char *lbm_last_error(const lbm_ctx *c);

/* Free the context and everything it allocated (NULL is ignored). */
void lbm_destroy(lbm_ctx *c);

/* LBM_ABI_VERSION of the library. */
int lbm_abi_version(void);

/* Observables without any allocation.  The paper has no counterpart: this serves callers
   that cannot let a library allocate device memory while they run -- code being recorded
   into a CUDA graph (cudaMalloc may not be called during stream capture), real-time loops
   that must not wait on the allocator, and applications whose own pool holds the whole
   device.  It computes what lbm_observables computes, for a state the caller holds:
     f       device pointer, FP64 populations after streaming, [n_species][9][nz][nx] (the
             layout lbm_get_fields writes), read on `stream`;
     p       the model parameters (host);
     out     device pointer to 16 + 9 nz + 2 nx doubles, written on `stream`: [0..1] mass,
             [2..3] momentum, [4] gamma, [5..6] wall force (bottom, top), [7] 1 if a density
             <= 0, NaN or Inf was met, [8..15] unused, then ux_z[nz], rho_z[2][nz], sxz_z[nz],
             fluid_z[nz], ps_x[nx], pxx_x[nx] (definitions as in lbm_obs; rho_z of species B
             is zero for one species), then the x-averages of the momentum mx_z[nz], mz_z[nz]
             and of the wall momentum exchange wallb_z[nz], wallt_z[nz] (nonzero on the first
             and last row).
   It allocates nothing: its scratch is one file-scope device array of
   LBM_NOALLOC_SCRATCH_BYTES that every GPU loading the library keeps until exit, which bounds
   the lattice: bytes needed = r256(nz*ceil(nx/32)*64) + r256(nx*ceil(nz/8)*16)
   + r256((nx+nz)*40) + 256, r256 rounding up to a multiple of 256 (a 1024 x 1024 lattice
   needs about 4.3 MB).  A call made outside a stream capture looks up the array's device
   address with the calling thread's current device (so a device reset is followed); a call
   made during a capture uses the address of the last lookup on that device, so make the first
   call on a device before any stream capture.  All calls share the
   array: calls that overlap on the GPU (other streams, other threads) race and must be
   serialised by the caller.  Asynchronous on `stream` (NULL = the default stream).
   Returns LBM_OK, LBM_EINVAL (NULL pointer or invalid description/parameters), LBM_ENOMEM
   (the lattice does not fit the fixed scratch) or LBM_ECUDA (no device / launch failure). */
#define LBM_NOALLOC_SCRATCH_BYTES (8u * 1024u * 1024u)
int lbm_observables_noalloc(const double *f, int nx, int nz, int n_species, int z_boundary,
                            const lbm_params *p, double *out, void *stream);

/* Batches (no counterpart in the paper: they serve sweeps over channel widths and drives, like
   the cooperative-length analysis of Sec. V).  The drive of lattice i of a batch: body force
   g along x and the wall velocities.  Defaults to the parameters' body_force and wall_u, and
   lbm_set_params resets every lattice to them.  Takes effect from the next step. */
int lbm_set_instance_drive(lbm_ctx *c, int i, double body_force, double wall_u_bottom, double wall_u_top);

/* Observables of lattice i of a batch (also valid for i = 0 of one lattice): the current state
   (averages = 0, synchronises and computes them) or the time averages sampled so far
   (averages != 0; reset with lbm_averages).  mass, momentum, wall_force and the z profiles
   (sized inst_nz[i]) are lattice i's; gamma, ps_x and pxx_x are left zero / untouched (the
   batch's column profiles average over all its lattices and are in lbm_observables). */
int lbm_instance_observables(lbm_ctx *c, int i, lbm_obs *out, int averages);

/* Autotuner (no counterpart in the paper).  Times the launch shapes of the PULL kernel on the
   context's own lattices -- depth 1 (one tile load in flight per CTA, 3 CTAs per SM in FP32) and
   depth 2 (two, 2 CTAs per SM) -- for `steps` steps each (1..10000), with observables every step
   if sampling is on and without otherwise, keeps the faster for that kind of pass (a context
   holds one shape for passes with observables and one for passes without; FP32 default: depth 1
   for both, FP64: depth 2), and puts the state, time sums and step count back, so the
   simulation does not advance.  chosen (may be NULL) receives the depth kept (0 for the other
   kernels, which have nothing to choose), ms_per_step[2] (may be NULL) the measured step times.
   Synchronises. */
int lbm_autotune(lbm_ctx *c, int steps, int *chosen, double *ms_per_step);

/* Tile shapes of the PULL kernel's step passes (no counterpart in the paper; they serve the
   batched sweeps of Sec. V).  A step pass runs tiles of 32 x 8 sites (one warp per tile row) or,
   in FP32, 64 x 8 (two warps per tile row: one CTA of 512 threads per SM, a halo of 304 instead
   of 2 x 176 psi/rho positions per 512 sites), at pipeline depth 1 or 2 (boxes in flight per
   CTA).  The shape changes which CTA does which sites and how much halo it reads, not the
   arithmetic: row sums stay per 32 columns and column sums per 8 rows, so states and observables
   are bit-identical across shapes.  lbm_autotune_tiles times `steps` (1..10000) steps of each
   (width, depth) in (32, 1), (32, 2), (64, 1), (64, 2) on the context's own lattices with the
   current sampling, keeps the fastest for that kind of pass (sampling on or off), and puts the
   state, time sums and step count back; *width and *depth (may be NULL) receive the choice,
   ms_per_step[4] (may be NULL) the milliseconds per step of the four (0 for width 64 in FP64,
   which has none).  Synchronises.  lbm_set_tile_shape sets a shape for both kinds of pass.  Both
   return LBM_EINVAL for the other kernels, and lbm_set_tile_shape for a width other than 32 / 64,
   a depth other than 1 / 2, or width 64 in FP64. */
int lbm_autotune_tiles(lbm_ctx *c, int steps, int *width, int *depth, double *ms_per_step);
int lbm_set_tile_shape(lbm_ctx *c, int width, int depth);

/* Self-test of failure detection (no counterpart in the paper).  The step kernels' only
   device-side waits are bounded waits on TMA copies; an expired wait sets a flag that the next
   synchronising call reports as LBM_ETIMEOUT, and the kernel leaves without faulting.  This
   runs the same bounded wait on a barrier that nothing completes, for `cycles` SM clock cycles
   (1 <= cycles <= 4e9), on the context's stream, then synchronises.  Returns LBM_ETIMEOUT
   (the expected result: the wait expired and was reported, the context stays usable), LBM_OK
   (the wait did not expire: a defect), LBM_EINVAL or LBM_ECUDA.  The flag is cleared again so
   that the context's later calls are unaffected. */
int lbm_selftest_wait(lbm_ctx *c, long long cycles);

/* Set the state from populations after streaming, f [n_species][9][nz][nx] FP64 (the layout
   lbm_get_fields writes): restores a state read earlier, e.g. a checkpoint of a run that is
   recomputed for its adjoint.  The values are not checked: a density <= 0 or a NaN shows as
   LBM_ENONFINITE after the next step.  FP32 contexts store deviations from the parameters'
   rho_ref when it is >= 0, else from the reference densities of the last lbm_set_fields
   (LBM_EINVAL if there was none).  Resets the step counter and the time averages.
   Synchronises. */
int lbm_set_populations(lbm_ctx *c, const double *f, int where);

/* Snapshots (exact checkpoints): lbm_snapshot copies the current state -- the populations in
   the context's internal layout and precision, the step counter and the FP32 reference
   densities -- into lbm_snapshot_bytes(c) bytes of device memory at dst (asynchronous).  The
   last 256 bytes are a tail that also records the writing context, a sequence number and the
   shape.  lbm_restore makes the snapshot at src the current state again, bit for bit, and
   resets the time averages: it reads the tail back (synchronises), so it is right whatever was
   written at src since, and it returns LBM_EINVAL when src holds no snapshot of a context of
   this shape and precision.
   lbm_restore_own is the asynchronous form for a snapshot this context wrote at src with its
   last lbm_snapshot there: the step counter and reference densities come from the context's
   record of that call (it keeps the latest 1024 addresses; other addresses fall back to
   lbm_restore), and a one-thread kernel compares the tail's writer and sequence number with
   the record.  If src was overwritten since (the buffer freed and reused, another snapshot),
   the next synchronising call returns LBM_EINVAL and the restored state must not be used. */
long long lbm_snapshot_bytes(const lbm_ctx *c);
int lbm_snapshot(lbm_ctx *c, void *dst);
int lbm_restore(lbm_ctx *c, const void *src);
int lbm_restore_own(lbm_ctx *c, const void *src);

/* The current state as populations after streaming, f [n_species][9][nz][nx] in device memory,
   double (LBM_FP64) or float (LBM_FP32) values: lbm_get_fields without the synchronisation and
   in a chosen precision.  Asynchronous. */
int lbm_export_state(lbm_ctx *c, void *f, int precision);

/* Discrete adjoint (no counterpart in the paper: it differentiates the step of Eq. LB with the
   forces of Eq. FORCE and Sec. IV so that the couplings, relaxation times, drive and initial
   densities can be fitted to target profiles like those of Sec. IV).  Single periodic lattices
   only (LBM_PERIODIC, n_instances <= 1), otherwise LBM_EINVAL.  The model parameters are the
   context's (lbm_set_params, and the drive of lbm_set_instance_drive for lattice 0); the
   context's own state is neither read nor changed by the adjoint calls.  All pointers are device
   memory on the context's device, used on the context's stream; the calls are asynchronous.
   `precision` (LBM_FP64 or LBM_FP32, independent of the context's) is the type of the state and
   adjoint arrays (double or float) and of their arithmetic; the parameter derivatives are
   accumulated in FP64 in both (per block in FP64 or double-float pairs, over blocks and steps
   in FP64).  A state array is [n_species][9][nz][nx] (the layout lbm_get_fields writes); an
   adjoint array lam = dJ/df has the same layout.  theta, the order of grad[8]: G1[A], G1[B],
   G2[A], G2[B], G_AB, tau[A], tau[B], body_force.

   lbm_record_states: for k = 0 .. nsteps - 1, writes the current state into states + k m
   (m = n_species 9 nz nx values of `precision`), then takes one step (as lbm_step): the states a
   backward sweep over these steps needs.  Asynchronous. */
int lbm_record_states(lbm_ctx *c, int nsteps, void *states, int precision);

/* One step back: for the step f_n -> f_{n+1} taken from the state f = f_n and lam_next =
   dJ/df_{n+1}, writes lam = dJ/df_n (must not overlap f or lam_next) and ADDS dJ/dtheta to
   grad[8]. */
int lbm_adjoint_step(lbm_ctx *c, const void *f, const void *lam_next, void *lam, double *grad, int precision);

/* nsteps steps back over the states recorded by lbm_record_states (states[k] = f_{n+k}): lam
   holds dJ/df_{n+nsteps} on entry and dJ/df_n on return (in place; the context keeps a second
   buffer); grad[8] += dJ/dtheta of those steps. */
int lbm_adjoint_steps(lbm_ctx *c, int nsteps, const void *states, void *lam, double *grad, int precision);

/* The calibration objective J = sum_z (ubar(z) - target_u[z])^2 + (rhobar_A(z) - target_rho[z])^2
   of the state f: ubar is the x-average of u = sum_s j_x,s / sum_s rho_s, rhobar_A the
   x-average of rho_A; target_u, target_rho hold nz doubles.  Writes J (one double, FP64 sums
   of the rows) and, unless dJdf is NULL, dJ/df (the layout and precision of f): the lam of the
   last state. */
int lbm_adjoint_objective(lbm_ctx *c, const void *f, const double *target_u, const double *target_rho,
                          double *J, void *dJdf, int precision);

/* For a run started by lbm_set_fields with u = NULL (populations W_l rho): the derivative with
   respect to those densities, g_rho [n_species][nz][nx] doubles = sum_l W_l lam0[s][l],
   lam0 = dJ/df_0 in `precision`. */
int lbm_adjoint_initial(lbm_ctx *c, const void *lam0, double *g_rho, int precision);

#ifdef __cplusplus
}
#endif
#endif
