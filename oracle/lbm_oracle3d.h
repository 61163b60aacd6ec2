/*
 * lbm_oracle3d.h -- plain FP64 CPU oracle of the three-dimensional extension of the two-belt
 * Shan-Chen lattice Boltzmann step (arXiv:1402.6019, Sec. II.B: "along the lines of" its
 * references).  TEST INFRASTRUCTURE: only tests/ may call it; it shares no code with the CUDA
 * path.  Arrays are C-contiguous FP64 with x fastest: a field is [nz][ny][nx], populations
 * [n_species][19][nz][ny][nx].  Calls return 0 on success, 1 for a bad argument, 3 when an
 * allocation fails.
 */
#ifndef LBM_ORACLE3D_H
#define LBM_ORACLE3D_H

typedef struct {
    double tau[2];       /* BGK relaxation time of each species (Eq. LB), > 1/2           */
    double G1[2];        /* attraction of Eq. FORCE on |c|^2 <= 4                          */
    double G2[2];        /* repulsion of Eq. FORCE on |c|^2 <= 8                           */
    double G_AB;         /* A-B cross repulsion (first belt)                              */
    double rho0[2];      /* psi = 1 - exp(-rho / rho0)                                     */
    double weight_norm;  /* scale of every interaction weight (1/3: Eq. BULK)             */
    double body_force;   /* acceleration g along x: F_s += rho_s g                        */
    int psi_form;        /* 0: psi = 1 - exp(-rho / rho0); 1: psi = rho                    */
    int zbc;             /* 0: periodic in z; 1: walls at z = -1/2 and nz - 1/2 (halfway
                            bounce-back with Ladd's moving-wall term, Sec. IV); psi and rho
                            beyond a wall are the mirror image of the fluid rows           */
    double wall_u[2];    /* x-velocity of the bottom and top walls                        */
} lbmref3_params;

typedef struct lbmref3 lbmref3;

/* The link set and weights: links[92][3] (|c|^2 = 1, 2, 3, 4, 5, 6, 8 in that order), the
   attraction, repulsion and cross weights by |c|^2 (index 0..8), the D3Q19 velocities
   c19[19][3] and rest weights w19[19].  Any pointer may be NULL; returns the link count. */
int lbmref3_tables(int *links, double *w_att, double *w_rep, double *w_cross, int *c19, double *w19);
/* D3Q19 equilibrium (Sec. II) of density rho and velocity u[3] into out19[19]. */
int lbmref3_feq(double rho, const double *u, double *out19);

int lbmref3_create(lbmref3 **out, int nx, int ny, int nz, int n_species, const lbmref3_params *p);
void lbmref3_destroy(lbmref3 *L);
int lbmref3_set_params(lbmref3 *L, const lbmref3_params *p);
/* Populations at equilibrium with u = 0 for densities rho [n_species][nz][ny][nx] (> 0). */
int lbmref3_set_fields(lbmref3 *L, const double *rho);
int lbmref3_set_populations(lbmref3 *L, const double *f);
/* psi [n_species][nz][ny][nx] and the total force F [n_species][3][nz][ny][nx] of the current
   state (Eq. FORCE, cross term, body force); either may be NULL. */
int lbmref3_site_fields(lbmref3 *L, double *psi, double *F);
int lbmref3_step(lbmref3 *L, int nsteps);
/* rho [n_species][nz][ny][nx], barycentric u [3][nz][ny][nx], populations; any may be NULL. */
int lbmref3_get(lbmref3 *L, double *rho, double *u, double *f);
long long lbmref3_step_count(const lbmref3 *L);

#endif
