/*
 * lbm_oracle.h -- TEST INFRASTRUCTURE. Not part of the product path.
 *
 * Plain FP64 CPU statement of one time step of the two-belt ("frustrated")
 * multirange Shan-Chen lattice Boltzmann model of Sbragaglia, Benzi, Bernaschi
 * and Succi (arXiv:1402.6019), single component or A/B mixture.  Only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark may call it; it shares
 * no code, header or table with the CUDA library.
 *
 * State: post-streaming (pre-collision) populations f[s][l][z][x], x fastest.
 * Lattice: D2Q9 for the kinetic part (Eq. LB), the 25-speed 5x5 block of Fig. 1
 * for the interaction (Eq. FORCE).  x is the stream-flow direction, z the
 * cross-flow direction (Sec. IV).
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { LBMREF_OK = 0, LBMREF_EINVAL = 1, LBMREF_ENOMEM = 3, LBMREF_ENONFINITE = 4 };
enum { LBMREF_PERIODIC = 0, LBMREF_BOUNCEBACK = 1 };
enum { LBMREF_PSI_EXP = 0, LBMREF_PSI_RHO = 1 };
enum { LBMREF_WEIGHTS_PAPER = 0, LBMREF_WEIGHTS_CHEM09 = 1 };
enum { LBMREF_WALL_MIRROR = 0, LBMREF_WALL_ZERO = 1 };

typedef struct lbmref_ctx lbmref_ctx;

typedef struct {
    double tau[2];       /* BGK relaxation time per species (Eq. LB), > 1/2          */
    double G1[2];        /* short-range (attractive) coupling per species, Eq. FORCE */
    double G2[2];        /* mid-range (repulsive) coupling per species, Eq. FORCE    */
    double G_AB;         /* A-B cross repulsion (Sec. IV)                            */
    int psi_form;        /* LBMREF_PSI_EXP: psi = 1 - exp(-rho/rho0); _RHO: psi = rho */
    double rho0[2];      /* rho0 of the exponential pseudopotential                  */
    int weight_preset;   /* LBMREF_WEIGHTS_PAPER or LBMREF_WEIGHTS_CHEM09            */
    double weight_norm;  /* multiplies every interaction weight; App. B tables have
                            e2 = 1, Eq. BULK implies e2 = c_s^2: default 1/3         */
    double body_force;   /* acceleration g along x: F_s += rho_s g                    */
    double wall_u[2];    /* x-velocity of the bottom (z=-1/2) and top (z=nz-1/2) wall */
    int psi_wall;        /* ghost rows beyond a wall: mirror of the fluid, or zero   */
} lbmref_params;

typedef struct {
    double mass[2];        /* sum of rho_s                                            */
    double momentum[2];    /* sum over sites and species of j_s + F_s/2               */
    double gamma;          /* sum over x of the z-averaged P_xx - P_zz (Eq. DIS1)     */
    double wall_force[2];  /* x-momentum given per step, per unit length, to the
                              bottom and top wall by bounce-back                       */
    int nonfinite;         /* 1 if any reduced value is NaN or Inf                     */
    /* optional profiles (caller-owned, NULL to skip) */
    double *ux_z;          /* [nz]     x-average of the barycentric u_x               */
    double *rho_z;         /* [ns][nz] x-average of rho_s                             */
    double *sxz_z;         /* [nz]     x-average of the shear stress S_xz             */
    double *fluid_z;       /* [nz]     fluidity (d ux_z/dz) / sxz_z (Eq. fluidity)    */
    double *ps_x;          /* [nx]     z-average of P_xx - P_zz                       */
    double *pxx_x;         /* [nx]     z-average of P_xx                              */
} lbmref_obs;

int  lbmref_create(lbmref_ctx **out, int nx, int nz, int n_species, int z_boundary);
int  lbmref_set_params(lbmref_ctx *c, const lbmref_params *p);
/* rho: [ns][nz][nx] (> 0); u: [2][nz][nx] or NULL for u = 0.  Sets f = f_eq(rho, u). */
int  lbmref_set_fields(lbmref_ctx *c, const double *rho, const double *u);
/* f: [ns][9][nz][nx] populations (any values; rho = sum f must stay > 0). */
int  lbmref_set_populations(lbmref_ctx *c, const double *f);
/* Any pointer may be NULL.  rho [ns][nz][nx]; u [2][nz][nx] barycentric
   (sum_s j_s + F_s/2)/sum_s rho_s; f [ns][9][nz][nx]. */
int  lbmref_get_fields(lbmref_ctx *c, double *rho, double *u, double *f);
int  lbmref_step(lbmref_ctx *c, int nsteps);
int  lbmref_observables(lbmref_ctx *c, lbmref_obs *o);
/* Per-site diagnostics of the current state, any pointer may be NULL:
   psi [ns][nz][nx]; F [ns][2][nz][nx] total force (intra + cross + body);
   sint [ns][3][nz][nx] interaction stress (xx, zz, xz) of each species (App. A);
   P [3][nz][nx] total pressure tensor (xx, zz, xz) as in Sec. III;
   sxz [nz][nx] shear stress S_xz. */
int  lbmref_site_fields(lbmref_ctx *c, double *psi, double *F, double *sint,
                        double *P, double *sxz);
long long lbmref_step_count(const lbmref_ctx *c);
void lbmref_destroy(lbmref_ctx *c);

/* Discrete adjoint of one step on a periodic lattice (EINVAL with walls), linearised at
   the context's current state f_n (set it with lbmref_set_populations): from
   lam_next = dJ/df_{n+1} [ns][9][nz][nx] it writes lam = dJ/df_n and adds to
   grad[LBMREF_NPARAM] the derivatives with respect to, in order: G1[A], G1[B], G2[A],
   G2[B], G_AB, tau[A], tau[B], body_force.  The state is left unchanged. */
enum { LBMREF_NPARAM = 8 };
int  lbmref_adjoint_step(lbmref_ctx *c, const double *lam_next, double *lam, double *grad);

/* Tables.  c25 [25][2] link vectors (row 0 unused); cq [9][2] and wq [9] D2Q9;
   wsh [3][9] interaction weights by |c|^2 for (attraction, repulsion, cross) under
   the given preset, before weight_norm. */
void lbmref_tables(int preset, int *c25, int *cq, double *wq, double *wsh);
/* Equilibrium of Sec. II for D2Q9 at (rho, ux, uz). */
void lbmref_feq(double rho, double ux, double uz, double *feq9);

#ifdef __cplusplus
}
#endif
#endif
