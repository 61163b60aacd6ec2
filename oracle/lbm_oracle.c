/*
 * lbm_oracle.c -- TEST INFRASTRUCTURE. Not part of the product path.
 *
 * Plain FP64 CPU oracle for the time step of the two-belt multirange Shan-Chen
 * lattice Boltzmann model (Sbragaglia, Benzi, Bernaschi, Succi, arXiv:1402.6019).
 * Every function below follows one passage of the paper, in the paper's order
 * (moments -> pseudopotential -> force -> shifted equilibrium -> BGK -> streaming),
 * with plain loops over the lattice and no blocking or fusion.  Where the paper is
 * silent the reading used is stated at the point of use.
 *
 * Used only by tests/, the smoke check and the CPU-baseline leg of bench.py.
 * Shares no code with the CUDA path.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Lattices                                                                   */
/* ------------------------------------------------------------------------- */

/* D2Q9 velocities c_0..c_8.  Sec. II uses a Gauss-Hermite velocity set without
   naming it; the order c1=(1,0) c2=(0,1) c3=(-1,0) c4=(0,-1) c5=(1,1) c6=(-1,1)
   c7=(-1,-1) c8=(1,-1) is the one for which Appendix A's pair identities hold
   (c5-c3 = c1-c7 = c13, c5-c4 = c2-c7 = c14, c2-c8 = c6-c4 = c15,
    c6-c1 = c3-c8 = c16). */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CZ[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WLB[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double CS2 = 1.0 / 3.0; /* c_s^2 of D2Q9 */

/* Interaction links l = 1..24 of the 25-speed lattice (Fig. 1), grouped by shell
   |c|^2 = 1 (l=1..4), 2 (5..8), 4 (9..12), 5 (13..20), 8 (21..24).  Links 1..8
   coincide with the D2Q9 set; c13..c16 are fixed by Appendix A; c17..c20 are
   their opposites. */
static const int LX[25] = {0, 1, 0, -1, 0, 1, -1, -1, 1, 2, 0, -2, 0,
                           2, 1, -1, -2, -2, -1, 1, 2, 2, -2, -2, 2};
static const int LZ[25] = {0, 0, 1, 0, -1, 1, 1, -1, -1, 0, 2, 0, -2,
                           1, 2, 2, 1, -1, -2, -2, -1, 2, 2, -2, -2};

/* Interaction weights by shell |c|^2 (index 0..8).  The paper prints only the
   constraints (App. B: e2 = 1, Eqs. 4sum and 6sum) and Eq. FORCE's ranges:
   attraction w over |c|^2 <= 4 (l = 1..12), repulsion p over |c|^2 <= 8
   (l = 1..24), both 6th-order isotropic.  w is the unique solution of
   {e2 = 1, 4sum, 6sum} with w(5) = w(8) = 0; p is the solution that is also
   8th-order isotropic.  The cross term uses the 4th-order first-belt set. */
static const double W_ATTR_PAPER[9] = {0, 4.0 / 15.0, 1.0 / 10.0, 0, 1.0 / 120.0, 0, 0, 0, 0};
static const double W_REP[9] = {0,           4.0 / 21.0, 4.0 / 45.0, 0, 1.0 / 60.0,
                                2.0 / 315.0, 0,          0,          1.0 / 5040.0};
static const double W_BELT1[9] = {0, 1.0 / 3.0, 1.0 / 12.0, 0, 0, 0, 0, 0, 0};

struct lbmref_ctx {
    int nx, nz, ns, zbc;
    lbmref_params p;
    double wa[9], wr[9], wc[9]; /* attraction, repulsion, cross weights by |c|^2 */
    int na;                     /* number of links carrying the attraction       */
    double *f, *fn;             /* [ns][9][nz][nx]                               */
    double *rho, *jx, *jz;      /* [ns][nz][nx]                                  */
    double *psi, *Fx, *Fz;      /* [ns][nz][nx]                                  */
    long long nstep;
};

static size_t site(const lbmref_ctx *c, int x, int z) { return (size_t)z * c->nx + x; }
static size_t nsites(const lbmref_ctx *c) { return (size_t)c->nx * c->nz; }
static double *pop(const lbmref_ctx *c, double *base, int s, int l) {
    return base + ((size_t)s * 9 + l) * nsites(c);
}
static int wrap(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}
/* Reflection of a row index about the wall planes z = -1/2 and z = nz - 1/2. */
static int mirror(int z, int n) {
    int m = z % (2 * n);
    if (m < 0) m += 2 * n;
    return m >= n ? 2 * n - 1 - m : m;
}

/* A per-site field read at (x, z), possibly beyond the domain: periodic in x;
   in z periodic, or (with walls) the ghost-row reading: mirror image of the fluid
   about the wall plane, or zero. */
static double field_at(const lbmref_ctx *c, const double *fld, int x, int z) {
    x = wrap(x, c->nx);
    if (c->zbc == LBMREF_PERIODIC) {
        z = wrap(z, c->nz);
    } else if (z < 0 || z >= c->nz) {
        if (c->p.psi_wall == LBMREF_WALL_ZERO) return 0.0;
        z = mirror(z, c->nz);
    }
    return fld[site(c, x, z)];
}

void lbmref_tables(int preset, int *c25, int *cq, double *wq, double *wsh) {
    if (c25)
        for (int l = 0; l < 25; ++l) {
            c25[2 * l] = LX[l];
            c25[2 * l + 1] = LZ[l];
        }
    if (cq)
        for (int l = 0; l < 9; ++l) {
            cq[2 * l] = CX[l];
            cq[2 * l + 1] = CZ[l];
        }
    if (wq)
        for (int l = 0; l < 9; ++l) wq[l] = WLB[l];
    if (wsh)
        for (int q = 0; q < 9; ++q) {
            wsh[q] = preset == LBMREF_WEIGHTS_CHEM09 ? W_BELT1[q] : W_ATTR_PAPER[q];
            wsh[9 + q] = W_REP[q];
            wsh[18 + q] = W_BELT1[q];
        }
}

/* Equilibrium of Sec. II: second moment c_s^2 rho delta + rho u u, truncated at
   second order in u (D2Q9 weights). */
void lbmref_feq(double rho, double ux, double uz, double *feq) {
    double usq = ux * ux + uz * uz;
    for (int l = 0; l < 9; ++l) {
        double cu = CX[l] * ux + CZ[l] * uz;
        feq[l] = WLB[l] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
    }
}

int lbmref_create(lbmref_ctx **out, int nx, int nz, int ns, int zbc) {
    if (!out || nx < 1 || nz < 1 || (ns != 1 && ns != 2) ||
        (zbc != LBMREF_PERIODIC && zbc != LBMREF_BOUNCEBACK))
        return LBMREF_EINVAL;
    lbmref_ctx *c = (lbmref_ctx *)calloc(1, sizeof *c);
    if (!c) return LBMREF_ENOMEM;
    c->nx = nx;
    c->nz = nz;
    c->ns = ns;
    c->zbc = zbc;
    size_t n = nsites(c);
    c->f = (double *)calloc((size_t)ns * 9 * n, sizeof(double));
    c->fn = (double *)calloc((size_t)ns * 9 * n, sizeof(double));
    c->rho = (double *)calloc((size_t)ns * n, sizeof(double));
    c->jx = (double *)calloc((size_t)ns * n, sizeof(double));
    c->jz = (double *)calloc((size_t)ns * n, sizeof(double));
    c->psi = (double *)calloc((size_t)ns * n, sizeof(double));
    c->Fx = (double *)calloc((size_t)ns * n, sizeof(double));
    c->Fz = (double *)calloc((size_t)ns * n, sizeof(double));
    if (!c->f || !c->fn || !c->rho || !c->jx || !c->jz || !c->psi || !c->Fx || !c->Fz) {
        lbmref_destroy(c);
        return LBMREF_ENOMEM;
    }
    lbmref_params d;
    memset(&d, 0, sizeof d);
    d.tau[0] = d.tau[1] = 1.0;
    d.rho0[0] = d.rho0[1] = 1.0;
    d.weight_norm = 1.0 / 3.0; /* Eq. BULK's c_s^2 normalisation (reading) */
    lbmref_set_params(c, &d);
    *out = c;
    return LBMREF_OK;
}

void lbmref_destroy(lbmref_ctx *c) {
    if (!c) return;
    free(c->f);
    free(c->fn);
    free(c->rho);
    free(c->jx);
    free(c->jz);
    free(c->psi);
    free(c->Fx);
    free(c->Fz);
    free(c);
}

int lbmref_set_params(lbmref_ctx *c, const lbmref_params *p) {
    if (!c || !p) return LBMREF_EINVAL;
    for (int s = 0; s < c->ns; ++s) {
        if (!(p->tau[s] > 0.5)) return LBMREF_EINVAL;
        if (p->psi_form == LBMREF_PSI_EXP && !(p->rho0[s] > 0.0)) return LBMREF_EINVAL;
    }
    if (p->psi_form != LBMREF_PSI_EXP && p->psi_form != LBMREF_PSI_RHO) return LBMREF_EINVAL;
    if (p->weight_preset != LBMREF_WEIGHTS_PAPER && p->weight_preset != LBMREF_WEIGHTS_CHEM09)
        return LBMREF_EINVAL;
    if (p->psi_wall != LBMREF_WALL_MIRROR && p->psi_wall != LBMREF_WALL_ZERO) return LBMREF_EINVAL;
    if (!(p->weight_norm > 0.0)) return LBMREF_EINVAL;
    c->p = *p;
    double wsh[27];
    lbmref_tables(p->weight_preset, NULL, NULL, NULL, wsh);
    for (int q = 0; q < 9; ++q) {
        c->wa[q] = p->weight_norm * wsh[q];
        c->wr[q] = p->weight_norm * wsh[9 + q];
        c->wc[q] = p->weight_norm * wsh[18 + q];
    }
    /* Eq. FORCE: attraction over l = 1..12; the CHEM09 reading over l = 1..8. */
    c->na = p->weight_preset == LBMREF_WEIGHTS_CHEM09 ? 8 : 12;
    return LBMREF_OK;
}

int lbmref_set_fields(lbmref_ctx *c, const double *rho, const double *u) {
    if (!c || !rho) return LBMREF_EINVAL;
    size_t n = nsites(c);
    for (size_t i = 0; i < (size_t)c->ns * n; ++i)
        if (!(rho[i] > 0.0) || !isfinite(rho[i])) return LBMREF_EINVAL;
    for (int s = 0; s < c->ns; ++s)
        for (int z = 0; z < c->nz; ++z)
            for (int x = 0; x < c->nx; ++x) {
                size_t i = site(c, x, z);
                double ux = u ? u[i] : 0.0, uz = u ? u[n + i] : 0.0;
                double feq[9];
                lbmref_feq(rho[s * n + i], ux, uz, feq);
                for (int l = 0; l < 9; ++l) pop(c, c->f, s, l)[i] = feq[l];
            }
    c->nstep = 0;
    return LBMREF_OK;
}

int lbmref_set_populations(lbmref_ctx *c, const double *f) {
    if (!c || !f) return LBMREF_EINVAL;
    memcpy(c->f, f, (size_t)c->ns * 9 * nsites(c) * sizeof(double));
    c->nstep = 0;
    return LBMREF_OK;
}

long long lbmref_step_count(const lbmref_ctx *c) { return c ? c->nstep : -1; }

/* ------------------------------------------------------------------------- */
/* The step, in the paper's order                                            */
/* ------------------------------------------------------------------------- */

/* Moments of Sec. II: rho = sum_l f_l, rho u = sum_l f_l c_l (per species). */
static void moments(lbmref_ctx *c) {
    size_t n = nsites(c);
    for (int s = 0; s < c->ns; ++s)
#pragma omp parallel for schedule(static)
        for (size_t i = 0; i < n; ++i) {
            double r = 0.0, jx = 0.0, jz = 0.0;
            for (int l = 0; l < 9; ++l) {
                double fl = pop(c, c->f, s, l)[i];
                r += fl;
                jx += fl * CX[l];
                jz += fl * CZ[l];
            }
            c->rho[s * n + i] = r;
            c->jx[s * n + i] = jx;
            c->jz[s * n + i] = jz;
        }
}

/* Pseudopotential of Sec. IV: psi(rho) = 1 - exp(-rho/rho0) (or psi = rho). */
static void pseudopotential(lbmref_ctx *c) {
    size_t n = nsites(c);
    for (int s = 0; s < c->ns; ++s)
#pragma omp parallel for schedule(static)
        for (size_t i = 0; i < n; ++i) {
            double r = c->rho[s * n + i];
            c->psi[s * n + i] =
                c->p.psi_form == LBMREF_PSI_EXP ? 1.0 - exp(-r / c->p.rho0[s]) : r;
        }
}

/* Total force on each species at each site:
   Eq. FORCE  F = -G1 psi(x) sum_{l=1..12} w(|c_l|^2) psi(x+c_l) c_l
                 -G2 psi(x) sum_{l=1..24} p(|c_l|^2) psi(x+c_l) c_l,
   plus the A-B cross repulsion of Sec. IV (formula not printed; reading: the
   first-belt Shan-Chen form with rho as the cross pseudopotential)
              F_s += -G_AB rho_s(x) sum_{l=1..8} w8(|c_l|^2) rho_s'(x+c_l) c_l,
   plus the volume force of Sec. IV read as an acceleration: F_s += rho_s g x. */
static void force(lbmref_ctx *c) {
    size_t n = nsites(c);
    for (int s = 0; s < c->ns; ++s) {
        const double *psi = c->psi + s * n;
#pragma omp parallel for schedule(static)
        for (int z = 0; z < c->nz; ++z)
            for (int x = 0; x < c->nx; ++x) {
                size_t i = site(c, x, z);
                double ax = 0.0, az = 0.0; /* short-range sum (weights w) */
                for (int l = 1; l <= c->na; ++l) {
                    double wl = c->wa[LX[l] * LX[l] + LZ[l] * LZ[l]];
                    double nb = field_at(c, psi, x + LX[l], z + LZ[l]);
                    ax += wl * nb * LX[l];
                    az += wl * nb * LZ[l];
                }
                double rx = 0.0, rz = 0.0; /* mid-range sum (weights p) */
                for (int l = 1; l <= 24; ++l) {
                    double wl = c->wr[LX[l] * LX[l] + LZ[l] * LZ[l]];
                    double nb = field_at(c, psi, x + LX[l], z + LZ[l]);
                    rx += wl * nb * LX[l];
                    rz += wl * nb * LZ[l];
                }
                double fx = -c->p.G1[s] * psi[i] * ax - c->p.G2[s] * psi[i] * rx;
                double fz = -c->p.G1[s] * psi[i] * az - c->p.G2[s] * psi[i] * rz;
                if (c->ns == 2) {
                    const double *rho_o = c->rho + (1 - s) * n;
                    double bx = 0.0, bz = 0.0;
                    for (int l = 1; l <= 8; ++l) {
                        double wl = c->wc[LX[l] * LX[l] + LZ[l] * LZ[l]];
                        double nb = field_at(c, rho_o, x + LX[l], z + LZ[l]);
                        bx += wl * nb * LX[l];
                        bz += wl * nb * LZ[l];
                    }
                    fx += -c->p.G_AB * c->rho[s * n + i] * bx;
                    fz += -c->p.G_AB * c->rho[s * n + i] * bz;
                }
                fx += c->rho[s * n + i] * c->p.body_force;
                c->Fx[s * n + i] = fx;
                c->Fz[s * n + i] = fz;
            }
    }
}

/* Shifted-velocity equilibrium and BGK relaxation of Eq. LB at one site and
   species: u_eq = u' + tau F / rho (Sec. II), with the common velocity
   u' = sum_s (j_s/tau_s) / sum_s (rho_s/tau_s) of the multicomponent model
   (reading; it is barycentric when all tau_s are equal).  Writes g_l. */
static void collide_site(const lbmref_ctx *c, int s, size_t i, double *g) {
    size_t n = nsites(c);
    double numx = 0.0, numz = 0.0, den = 0.0;
    for (int k = 0; k < c->ns; ++k) {
        numx += c->jx[k * n + i] / c->p.tau[k];
        numz += c->jz[k * n + i] / c->p.tau[k];
        den += c->rho[k * n + i] / c->p.tau[k];
    }
    double r = c->rho[s * n + i], tau = c->p.tau[s];
    double uex = numx / den + tau * c->Fx[s * n + i] / r;
    double uez = numz / den + tau * c->Fz[s * n + i] / r;
    double feq[9];
    lbmref_feq(r, uex, uez, feq);
    for (int l = 0; l < 9; ++l) {
        double fl = pop(c, c->f, s, l)[i];
        g[l] = fl - (fl - feq[l]) / tau;
    }
}

/* Streaming of Eq. LB, f_l(x + c_l, t+1) = g_l(x, t): periodic in x; in z
   periodic or halfway bounce-back on walls at z = -1/2 and z = nz - 1/2 moving
   along x at wall_u (Sec. IV's no-slip and +-U_w walls; reading: Ladd's moving-wall
   term with the local density, f_lbar(x) = g_l(x) - 2 W_l rho (c_l . U_w)/c_s^2).
   Adds the x-momentum each wall receives to wall[2] when wall != NULL. */
static void stream_site(const lbmref_ctx *c, int s, int x, int z, const double *g, double *fn,
                        double *wall) {
    size_t n = nsites(c);
    double r = c->rho[s * n + site(c, x, z)];
    for (int l = 0; l < 9; ++l) {
        int xd = wrap(x + CX[l], c->nx);
        int zd = z + CZ[l];
        if (c->zbc == LBMREF_PERIODIC) {
            zd = wrap(zd, c->nz);
        } else if (zd < 0 || zd >= c->nz) {
            int w = zd < 0 ? 0 : 1;
            double back = g[l] - 2.0 * WLB[l] * r * (CX[l] * c->p.wall_u[w]) / CS2;
            if (fn) pop(c, fn, s, OPP[l])[site(c, x, z)] = back;
            if (wall) wall[w] += CX[l] * (g[l] + back);
            continue;
        }
        if (fn) pop(c, fn, s, l)[site(c, xd, zd)] = g[l];
    }
}

static void collide_and_stream(lbmref_ctx *c) {
    /* every destination population is written by exactly one source site */
    for (int s = 0; s < c->ns; ++s)
#pragma omp parallel for schedule(static)
        for (int z = 0; z < c->nz; ++z)
            for (int x = 0; x < c->nx; ++x) {
                double g[9];
                collide_site(c, s, site(c, x, z), g);
                stream_site(c, s, x, z, g, c->fn, NULL);
            }
    double *t = c->f;
    c->f = c->fn;
    c->fn = t;
}

static void prepare(lbmref_ctx *c) {
    moments(c);
    pseudopotential(c);
    force(c);
}

int lbmref_step(lbmref_ctx *c, int nsteps) {
    if (!c || nsteps < 0) return LBMREF_EINVAL;
    for (int t = 0; t < nsteps; ++t) {
        prepare(c);
        collide_and_stream(c);
        c->nstep++;
    }
    return LBMREF_OK;
}

int lbmref_get_fields(lbmref_ctx *c, double *rho, double *u, double *f) {
    if (!c) return LBMREF_EINVAL;
    size_t n = nsites(c);
    prepare(c);
    if (rho) memcpy(rho, c->rho, (size_t)c->ns * n * sizeof(double));
    if (u)
        for (size_t i = 0; i < n; ++i) {
            double mx = 0.0, mz = 0.0, rt = 0.0;
            for (int s = 0; s < c->ns; ++s) {
                mx += c->jx[s * n + i] + 0.5 * c->Fx[s * n + i];
                mz += c->jz[s * n + i] + 0.5 * c->Fz[s * n + i];
                rt += c->rho[s * n + i];
            }
            u[i] = mx / rt;
            u[n + i] = mz / rt;
        }
    if (f) memcpy(f, c->f, (size_t)c->ns * 9 * n * sizeof(double));
    return LBMREF_OK;
}

/* ------------------------------------------------------------------------- */
/* Stress (Sec. III and Appendix A)                                          */
/* ------------------------------------------------------------------------- */

/* Interaction stress of one species at one site, Appendix A, for one coupling
   G with weights W over links 1..nl: the shells |c|^2 = 1, 2 (node products),
   4 and 8 (node and half-link products psi(x - c/2) psi(x + c/2)) and 5 (node
   products and the c13..c16 pair terms).  Adds (xx, zz, xz) into out[3]. */
static void shell_stress(const lbmref_ctx *c, const double *psi, int x, int z, double G,
                         const double *W, int nl, double *out) {
    double p0 = field_at(c, psi, x, z);
    for (int l = 1; l <= nl; ++l) {
        int q = LX[l] * LX[l] + LZ[l] * LZ[l];
        double wl = W[q];
        if (wl == 0.0) continue;
        double pr; /* the psi products carried by link l */
        double pref = (q == 1 || q == 2) ? G / 2.0 : G / 4.0;
        pr = p0 * field_at(c, psi, x + LX[l], z + LZ[l]);
        if (q == 4 || q == 8)
            pr += field_at(c, psi, x - LX[l] / 2, z - LZ[l] / 2) *
                  field_at(c, psi, x + LX[l] / 2, z + LZ[l] / 2);
        out[0] += pref * wl * pr * LX[l] * LX[l];
        out[1] += pref * wl * pr * LZ[l] * LZ[l];
        out[2] += pref * wl * pr * LX[l] * LZ[l];
    }
    if (nl >= 20 && W[5] != 0.0) {
        /* pair terms of sigma^(5): psi(x+ca) psi(x+cb) with ca - cb = c13..c16 */
        static const int PA[4][4] = {{5, 3, 1, 7}, {5, 4, 2, 7}, {2, 8, 6, 4}, {6, 1, 3, 8}};
        for (int k = 0; k < 4; ++k) {
            int l = 13 + k;
            double pr = field_at(c, psi, x + CX[PA[k][0]], z + CZ[PA[k][0]]) *
                            field_at(c, psi, x + CX[PA[k][1]], z + CZ[PA[k][1]]) +
                        field_at(c, psi, x + CX[PA[k][2]], z + CZ[PA[k][2]]) *
                            field_at(c, psi, x + CX[PA[k][3]], z + CZ[PA[k][3]]);
            out[0] += G / 4.0 * W[5] * pr * LX[l] * LX[l];
            out[1] += G / 4.0 * W[5] * pr * LZ[l] * LZ[l];
            out[2] += G / 4.0 * W[5] * pr * LX[l] * LZ[l];
        }
    }
}

/* Cross-species stress, first belt (reading, by analogy with sigma^(1), sigma^(2):
   the pair product psi(x)psi(x+c) of one species becomes
   rho_A(x) rho_B(x+c) + rho_B(x) rho_A(x+c)). */
static void cross_stress(const lbmref_ctx *c, int x, int z, double *out) {
    size_t n = nsites(c);
    const double *ra = c->rho, *rb = c->rho + n;
    double a0 = field_at(c, ra, x, z), b0 = field_at(c, rb, x, z);
    for (int l = 1; l <= 8; ++l) {
        double wl = c->wc[LX[l] * LX[l] + LZ[l] * LZ[l]];
        double pr = a0 * field_at(c, rb, x + LX[l], z + LZ[l]) +
                    b0 * field_at(c, ra, x + LX[l], z + LZ[l]);
        out[0] += c->p.G_AB / 2.0 * wl * pr * LX[l] * LX[l];
        out[1] += c->p.G_AB / 2.0 * wl * pr * LZ[l] * LZ[l];
        out[2] += c->p.G_AB / 2.0 * wl * pr * LX[l] * LZ[l];
    }
}

/* Per-site stresses of the current (prepared) state.
   sint_s: interaction stress of species s (App. A, both couplings).
   P: pressure tensor of Sec. III, summed over species,
      P_ij = sum_s [c_s^2 rho_s delta_ij + sint_s,ij + (tau_s - 1/2)^2 F_s,i F_s,j / rho_s]
             + sigma^AB_ij.
   S_xz: shear stress (reading; the paper only names "the stress"): minus the xz momentum flux
      of the lattice, kinetic and interaction,
      S_xz = -sum_s (1/2) sum_l (f_l,s + g_l,s) c_lx c_lz - [ sum_s sint_s,xz + sigma^AB_xz ],
      with g the post-collision populations of Eq. LB (collide_site).  The kinetic part is the
      second moment averaged over the collision: the populations that cross the lattice lines
      around x are the ones streamed into x (f) and out of x (g), so at a steady state the row
      sums of S_xz equal the x-momentum that crosses the rows above and below (Eq. MECHANICAL's
      balance), including the drift of each species and the forcing of Sec. II.
   u: the barycentric velocity (sum_s j_s + F_s/2) / sum_s rho_s. */
static void site_stress(const lbmref_ctx *c, int x, int z, double sint[2][3], double P[3],
                        double *Sxz, double u[2]) {
    size_t n = nsites(c), i = site(c, x, z);
    double cr[3] = {0.0, 0.0, 0.0};
    P[0] = P[1] = P[2] = 0.0;
    double mx = 0.0, mz = 0.0, rt = 0.0;
    for (int s = 0; s < c->ns; ++s) {
        sint[s][0] = sint[s][1] = sint[s][2] = 0.0;
        shell_stress(c, c->psi + s * n, x, z, c->p.G1[s], c->wa, c->na, sint[s]);
        shell_stress(c, c->psi + s * n, x, z, c->p.G2[s], c->wr, 24, sint[s]);
        double r = c->rho[s * n + i], fx = c->Fx[s * n + i], fz = c->Fz[s * n + i];
        double k2 = (c->p.tau[s] - 0.5) * (c->p.tau[s] - 0.5);
        P[0] += CS2 * r + sint[s][0] + k2 * fx * fx / r;
        P[1] += CS2 * r + sint[s][1] + k2 * fz * fz / r;
        P[2] += sint[s][2] + k2 * fx * fz / r;
        mx += c->jx[s * n + i] + 0.5 * fx;
        mz += c->jz[s * n + i] + 0.5 * fz;
        rt += r;
    }
    if (c->ns == 2) {
        cross_stress(c, x, z, cr);
        P[0] += cr[0];
        P[1] += cr[1];
        P[2] += cr[2];
    }
    u[0] = mx / rt;
    u[1] = mz / rt;
    double kin = 0.0, sint_xz = cr[2];
    for (int s = 0; s < c->ns; ++s) {
        double g[9];
        collide_site(c, s, i, g);
        for (int l = 0; l < 9; ++l) kin += 0.5 * (pop(c, c->f, s, l)[i] + g[l]) * CX[l] * CZ[l];
        sint_xz += sint[s][2];
    }
    *Sxz = -kin - sint_xz;
}

int lbmref_site_fields(lbmref_ctx *c, double *psi, double *F, double *sint, double *P,
                       double *sxz) {
    if (!c) return LBMREF_EINVAL;
    size_t n = nsites(c);
    prepare(c);
    if (psi) memcpy(psi, c->psi, (size_t)c->ns * n * sizeof(double));
    if (F)
        for (int s = 0; s < c->ns; ++s) {
            memcpy(F + (2 * s) * n, c->Fx + s * n, n * sizeof(double));
            memcpy(F + (2 * s + 1) * n, c->Fz + s * n, n * sizeof(double));
        }
    if (sint || P || sxz)
        for (int z = 0; z < c->nz; ++z)
            for (int x = 0; x < c->nx; ++x) {
                size_t i = site(c, x, z);
                double si[2][3], Pi[3], S, u[2];
                site_stress(c, x, z, si, Pi, &S, u);
                if (sint)
                    for (int s = 0; s < c->ns; ++s)
                        for (int k = 0; k < 3; ++k) sint[(3 * s + k) * n + i] = si[s][k];
                if (P)
                    for (int k = 0; k < 3; ++k) P[k * n + i] = Pi[k];
                if (sxz) sxz[i] = S;
            }
    return LBMREF_OK;
}

/* ------------------------------------------------------------------------- */
/* Observables (Secs. III-IV)                                                */
/* ------------------------------------------------------------------------- */

int lbmref_observables(lbmref_ctx *c, lbmref_obs *o) {
    if (!c || !o) return LBMREF_EINVAL;
    int nx = c->nx, nz = c->nz;
    size_t n = nsites(c);
    prepare(c);
    double *ux = (double *)calloc((size_t)nz, sizeof(double));
    double *sx = (double *)calloc((size_t)nz, sizeof(double));
    double *rz = (double *)calloc((size_t)2 * nz, sizeof(double));
    double *ps = (double *)calloc((size_t)nx, sizeof(double));
    double *px = (double *)calloc((size_t)nx, sizeof(double));
    if (!ux || !sx || !rz || !ps || !px) {
        free(ux); free(sx); free(rz); free(ps); free(px);
        return LBMREF_ENOMEM;
    }
    double mass[2] = {0.0, 0.0}, mom[2] = {0.0, 0.0}, wall[2] = {0.0, 0.0};
    for (int z = 0; z < nz; ++z)
        for (int x = 0; x < nx; ++x) {
            size_t i = site(c, x, z);
            double si[2][3], P[3], S, u[2];
            site_stress(c, x, z, si, P, &S, u);
            for (int s = 0; s < c->ns; ++s) {
                mass[s] += c->rho[s * n + i];
                mom[0] += c->jx[s * n + i] + 0.5 * c->Fx[s * n + i];
                mom[1] += c->jz[s * n + i] + 0.5 * c->Fz[s * n + i];
                rz[s * nz + z] += c->rho[s * n + i];
                if (c->zbc == LBMREF_BOUNCEBACK && (z == 0 || z == nz - 1)) {
                    double g[9];
                    collide_site(c, s, i, g);
                    stream_site(c, s, x, z, g, NULL, wall);
                }
            }
            ux[z] += u[0];
            sx[z] += S;
            ps[x] += P[0] - P[1];
            px[x] += P[0];
        }
    for (int z = 0; z < nz; ++z) {
        ux[z] /= nx;
        sx[z] /= nx;
        for (int s = 0; s < c->ns; ++s) rz[s * nz + z] /= nx;
    }
    double gamma = 0.0;
    for (int x = 0; x < nx; ++x) {
        ps[x] /= nz;
        px[x] /= nz;
        gamma += ps[x];
    }
    for (int s = 0; s < 2; ++s) o->mass[s] = s < c->ns ? mass[s] : 0.0;
    o->momentum[0] = mom[0];
    o->momentum[1] = mom[1];
    o->gamma = gamma;
    o->wall_force[0] = wall[0] / nx;
    o->wall_force[1] = wall[1] / nx;
    int bad = !isfinite(gamma) || !isfinite(mom[0]) || !isfinite(mom[1]);
    for (int s = 0; s < c->ns; ++s) bad |= !isfinite(mass[s]);
    o->nonfinite = bad;
    if (o->ux_z) memcpy(o->ux_z, ux, (size_t)nz * sizeof(double));
    if (o->sxz_z) memcpy(o->sxz_z, sx, (size_t)nz * sizeof(double));
    if (o->rho_z) memcpy(o->rho_z, rz, (size_t)c->ns * nz * sizeof(double));
    if (o->ps_x) memcpy(o->ps_x, ps, (size_t)nx * sizeof(double));
    if (o->pxx_x) memcpy(o->pxx_x, px, (size_t)nx * sizeof(double));
    if (o->fluid_z)
        /* Eq. fluidity: f = (shear rate)/(stress), with the shear rate the central
           difference of ux_z (one-sided at the wall rows, wrapped when periodic). */
        for (int z = 0; z < nz; ++z) {
            double gd;
            if (nz == 1)
                gd = 0.0;
            else if (c->zbc == LBMREF_PERIODIC)
                gd = 0.5 * (ux[wrap(z + 1, nz)] - ux[wrap(z - 1, nz)]);
            else if (z == 0)
                gd = ux[1] - ux[0];
            else if (z == nz - 1)
                gd = ux[nz - 1] - ux[nz - 2];
            else
                gd = 0.5 * (ux[z + 1] - ux[z - 1]);
            o->fluid_z[z] = gd / sx[z];
        }
    free(ux); free(sx); free(rz); free(ps); free(px);
    return LBMREF_OK;
}

/* ------------------------------------------------------------------------- */
/* Discrete adjoint of one step (periodic lattice)                           */
/* ------------------------------------------------------------------------- */

/* Vector-Jacobian product of one step f_n -> f_{n+1} = S(f_n; theta) at the state
   held by the context: given lam_next = dJ/df_{n+1}, writes lam = dJ/df_n and adds
   dJ/dtheta to grad[LBMREF_NPARAM] (G1[A], G1[B], G2[A], G2[B], G_AB, tau[A], tau[B],
   body_force).  Each forward stage of the step (moments, pseudopotential, force,
   common velocity, shifted equilibrium, relaxation, streaming) is differentiated by
   hand and applied in reverse order, with plain loops and the neighbour terms of
   the force scattered back to the neighbours they came from. */
int lbmref_adjoint_step(lbmref_ctx *c, const double *lam_next, double *lam, double *grad) {
    if (!c || !lam_next || !lam || !grad) return LBMREF_EINVAL;
    if (c->zbc != LBMREF_PERIODIC) return LBMREF_EINVAL;
    const size_t n = nsites(c);
    const int ns = c->ns;
    prepare(c); /* rho, j, psi, F of the state f_n */
    double *mu = calloc((size_t)ns * 9 * n, sizeof(double));  /* dJ/d(post-collision) */
    double *dF = calloc((size_t)ns * 2 * n, sizeof(double));  /* dJ/dF_s (x, z)       */
    double *drho = calloc((size_t)ns * n, sizeof(double));    /* dJ/drho_s            */
    double *dpsi = calloc((size_t)ns * n, sizeof(double));    /* dJ/dpsi_s            */
    double *djx = calloc((size_t)ns * n, sizeof(double));     /* dJ/dj_s              */
    double *djz = calloc((size_t)ns * n, sizeof(double));
    if (!mu || !dF || !drho || !dpsi || !djx || !djz) {
        free(mu), free(dF), free(drho), free(dpsi), free(djx), free(djz);
        return LBMREF_ENOMEM;
    }
    /* streaming, transposed: the post-collision g_l(x) became f_l(x + c_l) */
    for (int s = 0; s < ns; ++s)
        for (int l = 0; l < 9; ++l)
            for (int z = 0; z < c->nz; ++z)
                for (int x = 0; x < c->nx; ++x)
                    pop(c, mu, s, l)[site(c, x, z)] =
                        lam_next[((size_t)s * 9 + l) * n + site(c, wrap(x + CX[l], c->nx), wrap(z + CZ[l], c->nz))];
    /* relaxation, equilibrium, shifted velocity, common velocity: site by site */
    for (size_t i = 0; i < n; ++i) {
        double numx = 0.0, numz = 0.0, den = 0.0;
        for (int k = 0; k < ns; ++k) {
            numx += c->jx[k * n + i] / c->p.tau[k];
            numz += c->jz[k * n + i] / c->p.tau[k];
            den += c->rho[k * n + i] / c->p.tau[k];
        }
        const double upx = numx / den, upz = numz / den;
        double dupx = 0.0, dupz = 0.0; /* dJ/du' */
        for (int s = 0; s < ns; ++s) {
            const double r = c->rho[s * n + i], tau = c->p.tau[s];
            const double Fx = c->Fx[s * n + i], Fz = c->Fz[s * n + i];
            const double ux = upx + tau * Fx / r, uz = upz + tau * Fz / r;
            double feq[9];
            lbmref_feq(r, ux, uz, feq);
            /* g_l = f_l - (f_l - feq_l)/tau */
            double dfeq[9];
            for (int l = 0; l < 9; ++l) {
                const double m = pop(c, mu, s, l)[i];
                const double fl = pop(c, c->f, s, l)[i];
                dfeq[l] = m / tau;
                grad[5 + s] += m * (fl - feq[l]) / (tau * tau);
            }
            /* feq_l = W_l rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u) */
            double ar = 0.0, aux = 0.0, auz = 0.0;
            for (int l = 0; l < 9; ++l) {
                const double cu = CX[l] * ux + CZ[l] * uz;
                ar += dfeq[l] * WLB[l] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uz * uz));
                aux += dfeq[l] * WLB[l] * r * (3.0 * CX[l] + 9.0 * cu * CX[l] - 3.0 * ux);
                auz += dfeq[l] * WLB[l] * r * (3.0 * CZ[l] + 9.0 * cu * CZ[l] - 3.0 * uz);
            }
            /* u_s = u' + tau F_s / rho_s */
            dupx += aux;
            dupz += auz;
            dF[(s * 2 + 0) * n + i] = aux * tau / r;
            dF[(s * 2 + 1) * n + i] = auz * tau / r;
            drho[s * n + i] += ar - (aux * Fx + auz * Fz) * tau / (r * r);
            grad[5 + s] += (aux * Fx + auz * Fz) / r;
        }
        /* u' = sum_k j_k / tau_k / sum_k rho_k / tau_k */
        const double dnx = dupx / den, dnz = dupz / den, dden = -(dupx * upx + dupz * upz) / den;
        for (int k = 0; k < ns; ++k) {
            const double tk = c->p.tau[k];
            djx[k * n + i] += dnx / tk;
            djz[k * n + i] += dnz / tk;
            drho[k * n + i] += dden / tk;
            grad[5 + k] += -(c->jx[k * n + i] * dnx + c->jz[k * n + i] * dnz + c->rho[k * n + i] * dden) / (tk * tk);
        }
    }
    /* the force of Eq. FORCE, the cross term and the drive, scattered back */
    for (int s = 0; s < ns; ++s) {
        const double *psi = c->psi + s * n;
        for (int z = 0; z < c->nz; ++z)
            for (int x = 0; x < c->nx; ++x) {
                const size_t i = site(c, x, z);
                const double bx = dF[(s * 2 + 0) * n + i], bz = dF[(s * 2 + 1) * n + i];
                const double r = c->rho[s * n + i];
                /* F = -G1 psi(x) sum w psi(x+c) c - G2 psi(x) sum p psi(x+c) c */
                double ax = 0.0, az = 0.0, rx = 0.0, rz = 0.0;
                for (int l = 1; l <= 24; ++l) {
                    const size_t j = site(c, wrap(x + LX[l], c->nx), wrap(z + LZ[l], c->nz));
                    const int q = LX[l] * LX[l] + LZ[l] * LZ[l];
                    const double bc = bx * LX[l] + bz * LZ[l];
                    const double wa = l <= c->na ? c->wa[q] : 0.0, wr = c->wr[q];
                    ax += wa * psi[j] * LX[l];
                    az += wa * psi[j] * LZ[l];
                    rx += wr * psi[j] * LX[l];
                    rz += wr * psi[j] * LZ[l];
                    dpsi[s * n + j] += -psi[i] * (c->p.G1[s] * wa + c->p.G2[s] * wr) * bc;
                }
                dpsi[s * n + i] += -(c->p.G1[s] * (bx * ax + bz * az) + c->p.G2[s] * (bx * rx + bz * rz));
                grad[0 + s] += -psi[i] * (bx * ax + bz * az);
                grad[2 + s] += -psi[i] * (bx * rx + bz * rz);
                /* cross: F_s += -G_AB rho_s(x) sum w8 rho_s'(x+c) c */
                if (ns == 2) {
                    const double *rho_o = c->rho + (1 - s) * n;
                    double cx = 0.0, cz = 0.0;
                    for (int l = 1; l <= 8; ++l) {
                        const size_t j = site(c, wrap(x + LX[l], c->nx), wrap(z + LZ[l], c->nz));
                        const double wl = c->wc[LX[l] * LX[l] + LZ[l] * LZ[l]];
                        cx += wl * rho_o[j] * LX[l];
                        cz += wl * rho_o[j] * LZ[l];
                        drho[(1 - s) * n + j] += -c->p.G_AB * r * wl * (bx * LX[l] + bz * LZ[l]);
                    }
                    drho[s * n + i] += -c->p.G_AB * (bx * cx + bz * cz);
                    grad[4] += -r * (bx * cx + bz * cz);
                }
                /* drive: F_s += rho_s g x */
                drho[s * n + i] += bx * c->p.body_force;
                grad[7] += r * bx;
            }
    }
    /* pseudopotential, then the moments rho = sum f, j = sum f c */
    for (int s = 0; s < ns; ++s)
        for (size_t i = 0; i < n; ++i) {
            const double r = c->rho[s * n + i];
            const double dpr = c->p.psi_form == LBMREF_PSI_EXP ? exp(-r / c->p.rho0[s]) / c->p.rho0[s] : 1.0;
            const double dr = drho[s * n + i] + dpr * dpsi[s * n + i];
            const double tau = c->p.tau[s];
            for (int l = 0; l < 9; ++l)
                lam[((size_t)s * 9 + l) * n + i] = (1.0 - 1.0 / tau) * pop(c, mu, s, l)[i] + dr +
                                                   djx[s * n + i] * CX[l] + djz[s * n + i] * CZ[l];
        }
    free(mu), free(dF), free(drho), free(dpsi), free(djx), free(djz);
    return LBMREF_OK;
}
