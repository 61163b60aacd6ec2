/*
 * lbm3d.h -- C ABI of the three-dimensional extension of the two-belt ("frustrated")
 * multirange Shan-Chen lattice Boltzmann step (arXiv:1402.6019).  The paper works in two
 * dimensions and leaves three to "the lines of" its references (Sec. II.B); this extension
 * carries the 2-D model's steps over:
 *  - D3Q19 populations with the equilibrium of Sec. II (rest weight 1/3, axis 1/18, edge 1/36,
 *    c_s^2 = 1/3), velocities in the order: rest, +x, -x, +y, -y, +z, -z, (1,1,0), (-1,-1,0),
 *    (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1), (0,1,1), (0,-1,-1), (0,1,-1),
 *    (0,-1,1) (each velocity followed by its opposite);
 *  - Eq. FORCE over the integer links of |c|^2 = 1, 2, 3, 4 (attraction G1, 32 links) and
 *    |c|^2 = 1, 2, 3, 4, 5, 6, 8 (repulsion G2, 92 links) with the weights that solve
 *    Appendix B's isotropy constraints in three dimensions (attraction 2/15, 1/15, 1/60, 1/120;
 *    repulsion 4/45, 1/21, 2/105, 5/504, 1/315, 1/630, 1/5040 by |c|^2), every weight scaled
 *    by weight_norm;
 *  - the A-B cross repulsion of Sec. IV over the 18 D3Q19 neighbours with weights 1/6, 1/12
 *    (|c|^2 = 1, 2), rho as the cross pseudopotential;
 *  - the shifted-velocity BGK collision of Sec. II with the common velocity
 *    u' = sum_s (j_s / tau_s) / sum_s (rho_s / tau_s) and u_s^eq = u' + tau_s F_s / rho_s, a body
 *    force rho_s g along x;
 *  - periodic in x and y; in z periodic or between walls at z = -1/2 and nz - 1/2 (halfway
 *    bounce-back with Ladd's moving-wall term for walls moving along x, Sec. IV), psi and rho
 *    beyond a wall the mirror image of the fluid rows.
 * Conventions as in lbm.h: status codes LBM_*, host arrays C-contiguous FP64 with x fastest
 * (a field is [nz][ny][nx], populations [n_species][19][nz][ny][nx]), "where" = LBM_HOST or
 * LBM_DEVICE (device memory on the context's device, used on its stream, owned by the
 * caller), calls enqueue on the context's stream and return unless they say they
 * synchronise; a context is bound to one device and stream and is not thread-safe.
 */
#ifndef LBM3D_H
#define LBM3D_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm3_ctx lbm3_ctx;

/* Lattice and execution description, fixed for the life of a context. */
typedef struct {
    int nx, ny, nz;   /* lattice sizes, each >= 1; nx * ny * nz <= 2^30                    */
    int n_species;    /* 1 or 2                                                            */
    int precision;    /* LBM_FP64 (plain FP64) or LBM_FP32 (FP32 deviations f - W_l rho_ref,s,
                         rho_ref,s the mean density of species s at lbm3_set_fields)         */
    int z_boundary;   /* LBM_PERIODIC or LBM_BOUNCEBACK                                     */
    int device;       /* CUDA device ordinal                                                */
    int pad_;
    void *stream;     /* cudaStream_t to run on, or NULL for a stream of the context's own  */
} lbm3_desc;

/* Defaults: 64^3, two species, FP32, periodic, device 0, own stream. */
void lbm3_default_desc(lbm3_desc *d);

/* Create a context (allocates its device memory).  LBM_EINVAL for a bad description,
   LBM_ECUDA without a usable device, LBM_ENOMEM when the memory does not fit. */
int lbm3_create(lbm3_ctx **out, const lbm3_desc *d);

/* Model parameters (the fields of lbm_params that the 3-D model has: tau, G1, G2, G_AB,
   psi_form, rho0, weight_norm, body_force, wall_u).  weight_preset must be
   LBM_WEIGHTS_PAPER and psi_wall LBM_WALL_MIRROR (the only 3-D readings); rho_ref as in lbm.h.
   LBM_EINVAL otherwise. */
int lbm3_set_params(lbm3_ctx *c, const lbm_params *p);

/* Populations at the equilibrium of Sec. II at rest for the densities rho
   [n_species][nz][ny][nx] (each > 0 and finite, else LBM_EINVAL).  Resets the step counter.
   Synchronises. */
int lbm3_set_fields(lbm3_ctx *c, const double *rho, int where);

/* The current state: rho [n_species][nz][ny][nx], the barycentric velocity
   u [3][nz][ny][nx] = (sum_s j_s + F_s / 2) / sum_s rho_s, and the post-streaming populations
   f [n_species][19][nz][ny][nx], FP64; any pointer may be NULL.  Synchronises. */
int lbm3_get_fields(lbm3_ctx *c, double *rho, double *u, double *f, int where);

/* nsteps (>= 0) time steps: a density pass (rho and psi into ghost-padded volumes), then the
   force, collision and streaming pass.  Asynchronous.  Captured into a caller's CUDA graph, the
   launches are recorded with their buffers and the context's host-side state (step counter, the
   current population buffer) advances as if they had run: replay such a graph once per capture. */
int lbm3_step(lbm3_ctx *c, int nsteps);

/* Totals of the current state: mass[s] = sum of rho_s (n_species entries), momentum[3] =
   the lattice momentum sum_s sum_l c_l f_l,s.  A site's sums over its 19 populations are formed
   in the context's precision (FP32 deviations: the sums the step forms rho with), the sums over
   the sites in FP64.  Synchronises. */
int lbm3_totals(lbm3_ctx *c, double *mass, double *momentum);

/* Advance nsteps >= 0 steps and, after each, write the totals of the new state into record i,
   the 5 doubles at (char *)dst + i * stride: mass A, mass B (zero for one species), the lattice
   momentum x, y, z.  They are the values lbm3_totals returns, summed in the same order, so the
   same bits.  dst is device memory or pinned host memory (cudaHostAlloc or registered); stride is
   a multiple of 8 bytes, at least 40.  The records are written by kernels on the context's
   stream: asynchronous, no host copy.  *ticket (may be NULL) receives the ticket of the run's last
   record (left as it is when nsteps is 0); lbm3_wait(c, ticket) waits until it and every record before it are written (an event;
   for one of the last 64 tickets, else the whole stream).  A failed step (density <= 0, NaN or
   Inf, a tile load that did not arrive) is reported by lbm3_synchronize, not here.  The next
   step's density pass forms each record along with its own work, so the populations are read once
   per step for both; lbm3_profile does not time these steps. */
int lbm3_step_totals(lbm3_ctx *c, int nsteps, double *dst, long long stride, long long *ticket);
int lbm3_wait(lbm3_ctx *c, long long ticket);

/* Wait for the context's stream; LBM_ENONFINITE if a step met a density <= 0, NaN or Inf,
   LBM_ETIMEOUT if a bounded device-side wait for a tile load gave up. */
int lbm3_synchronize(lbm3_ctx *c);

/* Kernel timing: while enabled, every launch of the two step kernels is bracketed by CUDA
   events; lbm3_profile_read returns their summed times in milliseconds (density pass,
   collide pass) and the steps timed since profiling was enabled.  Both synchronise. */
int lbm3_profile(lbm3_ctx *c, int enable);
int lbm3_profile_read(lbm3_ctx *c, double *ms, long long *steps);

/* Tile shapes of the collide pass: 0 = 32 x 4 x 2 sites (the default), 1 = 32 x 2 x 4,
   2 = 32 x 8 x 1 (256 threads each), 3 = 32 x 4 x 4 (512 threads).  The shape changes which
   CTA does which sites and how much of the psi / rho halo each reads, not the arithmetic:
   results are bit-identical.  lbm3_autotune times `steps` (1 .. 10000) steps of each shape on
   the context's own lattice, keeps the fastest, and puts the state and step counter back as
   they were; *chosen (may be NULL) receives the shape, ms[4] (may be NULL) the milliseconds per
   step of each.  Synchronises.  lbm3_set_shape sets a shape directly (LBM_EINVAL outside 0..3). */
int lbm3_autotune(lbm3_ctx *c, int steps, int *chosen, double *ms);
int lbm3_set_shape(lbm3_ctx *c, int shape);

/* One-line description of the last failure on c (or of the last lbm3_create failure when
   c is NULL). */
const char *lbm3_last_error(const lbm3_ctx *c);

/* Free the context and its device memory (NULL is ignored). */
void lbm3_destroy(lbm3_ctx *c);

#ifdef __cplusplus
}
#endif
#endif
