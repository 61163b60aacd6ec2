/*
 * lbm_oracle3d.c -- plain FP64 CPU oracle of the three-dimensional extension of the two-belt
 * ("frustrated") Shan-Chen lattice Boltzmann step of Sbragaglia, Benzi, Bernaschi and Succi
 * (arXiv:1402.6019).  TEST INFRASTRUCTURE: used only by tests/; it shares no code with the
 * CUDA path and is written for clarity, not speed.
 *
 * The paper works in two dimensions and leaves three to "the lines of" its references
 * (Sec. II.B, competing interactions).  This file takes the 2-D model's steps to three
 * dimensions with the same readings:
 *  - lattice: D3Q19 (rest, 6 axis, 12 edge velocities; weights 1/3, 1/18, 1/36; c_s^2 = 1/3),
 *    Eq. LB with the equilibrium of Sec. II, periodic in x and y, and in z or between walls
 *    (halfway bounce-back with Ladd's moving-wall term, psi and rho mirrored beyond a wall, as
 *    in two dimensions);
 *  - Eq. FORCE over the integer links of |c|^2 = 1, 2, 3, 4 (attraction, G1, 32 links) and
 *    |c|^2 = 1, 2, 3, 4, 5, 6, 8 (repulsion, G2, 92 links), with the weights that solve
 *    Appendix B's constraints in three dimensions: attraction e2 = 1 and isotropic to 6th order,
 *    repulsion e2 = 1 and isotropic to 8th order (each the unique solution on its shells);
 *  - A-B cross repulsion over the first belt (the 18 D3Q19 neighbours) with the 4th-order
 *    isotropic weights (1/6, 1/12), rho as the cross pseudopotential;
 *  - every interaction weight scaled by weight_norm (1/3: Eq. BULK);
 *  - shifted-velocity BGK of Sec. II with the common velocity u' = sum_s (j_s / tau_s) /
 *    sum_s (rho_s / tau_s), u_s^eq = u' + tau_s F_s / rho_s; body force g along x.
 * Loops run in a fixed order; no FMA contraction (built with -ffp-contract=off).  OpenMP splits
 * only loops whose iterations are independent (per site, or per destination row of the
 * streaming), so the results are the same for every thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "lbm_oracle3d.h"

/* D3Q19 velocities: rest, the 6 axis directions, the 12 edge directions. */
static const int C19[19][3] = {{0, 0, 0},   {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                               {0, 0, 1},   {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                               {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                               {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double w19(int l) { return l == 0 ? 1.0 / 3.0 : (l <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

/* the velocity opposite to c_l */
static int opp19(int l) {
    for (int m = 0; m < 19; ++m)
        if (C19[m][0] == -C19[l][0] && C19[m][1] == -C19[l][1] && C19[m][2] == -C19[l][2]) return m;
    return 0;
}

/* Interaction weights by shell |c|^2 (index 0..8; zero where the shell is not used). */
static const double W_ATT[9] = {0, 2.0 / 15.0, 1.0 / 15.0, 1.0 / 60.0, 1.0 / 120.0, 0, 0, 0, 0};
static const double W_REP[9] = {0, 4.0 / 45.0, 1.0 / 21.0, 2.0 / 105.0, 5.0 / 504.0, 1.0 / 315.0, 1.0 / 630.0, 0,
                                1.0 / 5040.0};
static const double W_CROSS[9] = {0, 1.0 / 6.0, 1.0 / 12.0, 0, 0, 0, 0, 0, 0};

#define NLINK 92
static int LINKS[NLINK][3];
static int nlinks_built = 0;

/* The links of Eq. FORCE in 3-D: every integer vector with |c|^2 in {1,...,8} (7 does not occur),
   in order of |c|^2, then of (x, y, z) from -2 upwards. */
static void build_links(void) {
    if (nlinks_built) return;
    int n = 0;
    for (int q = 1; q <= 8; ++q)
        for (int x = -2; x <= 2; ++x)
            for (int y = -2; y <= 2; ++y)
                for (int z = -2; z <= 2; ++z)
                    if (x * x + y * y + z * z == q) {
                        LINKS[n][0] = x;
                        LINKS[n][1] = y;
                        LINKS[n][2] = z;
                        ++n;
                    }
    nlinks_built = n;
}

struct lbmref3 {
    int nx, ny, nz, ns;
    long long n;
    lbmref3_params p;
    double *f, *ftmp;  /* [ns][19][nz][ny][nx] */
    long long steps;
};

static long long idx(const lbmref3 *L, int x, int y, int z) {
    x = ((x % L->nx) + L->nx) % L->nx;
    y = ((y % L->ny) + L->ny) % L->ny;
    z = ((z % L->nz) + L->nz) % L->nz;
    return ((long long)z * L->ny + y) * L->nx + x;
}

/* The site whose psi / rho a neighbour at height z reads: periodic in z, or with walls the
   mirror image about the wall plane (z = -1 reads row 0, z = -2 row 1; likewise at the top). */
static long long nbr(const lbmref3 *L, int x, int y, int z) {
    if (L->p.zbc) {
        if (z < 0) z = -1 - z;
        if (z >= L->nz) z = 2 * L->nz - 1 - z;
    }
    return idx(L, x, y, z);
}

static double psi_of(const lbmref3 *L, int s, double rho) {
    return L->p.psi_form == 1 ? rho : 1.0 - exp(-rho / L->p.rho0[s]);
}

int lbmref3_tables(int *links, double *w_att, double *w_rep, double *w_cross, int *c19, double *w19_out) {
    build_links();
    if (links) memcpy(links, LINKS, sizeof LINKS);
    if (w_att) memcpy(w_att, W_ATT, sizeof W_ATT);
    if (w_rep) memcpy(w_rep, W_REP, sizeof W_REP);
    if (w_cross) memcpy(w_cross, W_CROSS, sizeof W_CROSS);
    if (c19) memcpy(c19, C19, sizeof C19);
    if (w19_out)
        for (int l = 0; l < 19; ++l) w19_out[l] = w19(l);
    return nlinks_built;
}

int lbmref3_create(lbmref3 **out, int nx, int ny, int nz, int ns, const lbmref3_params *p) {
    if (!out || nx < 1 || ny < 1 || nz < 1 || (ns != 1 && ns != 2) || !p) return 1;
    build_links();
    lbmref3 *L = (lbmref3 *)calloc(1, sizeof *L);
    if (!L) return 3;
    L->nx = nx;
    L->ny = ny;
    L->nz = nz;
    L->ns = ns;
    L->n = (long long)nx * ny * nz;
    L->p = *p;
    L->f = (double *)calloc((size_t)(ns * 19 * L->n), sizeof(double));
    L->ftmp = (double *)calloc((size_t)(ns * 19 * L->n), sizeof(double));
    if (!L->f || !L->ftmp) {
        free(L->f);
        free(L->ftmp);
        free(L);
        return 3;
    }
    *out = L;
    return 0;
}

void lbmref3_destroy(lbmref3 *L) {
    if (!L) return;
    free(L->f);
    free(L->ftmp);
    free(L);
}

int lbmref3_set_params(lbmref3 *L, const lbmref3_params *p) {
    if (!L || !p) return 1;
    L->p = *p;
    return 0;
}

/* Equilibrium of Sec. II for D3Q19. */
static double feq(int l, double rho, const double u[3]) {
    const double cu = C19[l][0] * u[0] + C19[l][1] * u[1] + C19[l][2] * u[2];
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return w19(l) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

int lbmref3_feq(double rho, const double *u, double *out19) {
    for (int l = 0; l < 19; ++l) out19[l] = feq(l, rho, u);
    return 0;
}

int lbmref3_set_fields(lbmref3 *L, const double *rho) {
    if (!L || !rho) return 1;
    const double u0[3] = {0.0, 0.0, 0.0};
    for (int s = 0; s < L->ns; ++s)
        for (long long i = 0; i < L->n; ++i) {
            const double r = rho[s * L->n + i];
            if (!(r > 0.0) || !isfinite(r)) return 1;
            for (int l = 0; l < 19; ++l) L->f[(s * 19 + l) * L->n + i] = feq(l, r, u0);
        }
    L->steps = 0;
    return 0;
}

int lbmref3_set_populations(lbmref3 *L, const double *f) {
    if (!L || !f) return 1;
    memcpy(L->f, f, sizeof(double) * (size_t)(L->ns * 19 * L->n));
    L->steps = 0;
    return 0;
}

static void moments(const lbmref3 *L, double *rho /*[ns][n]*/, double *j /*[ns][3][n]*/) {
    for (int s = 0; s < L->ns; ++s)
#pragma omp parallel for schedule(static)
        for (long long i = 0; i < L->n; ++i) {
            double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
            for (int l = 0; l < 19; ++l) {
                const double v = L->f[(s * 19 + l) * L->n + i];
                r += v;
                jx += v * C19[l][0];
                jy += v * C19[l][1];
                jz += v * C19[l][2];
            }
            rho[s * L->n + i] = r;
            j[(s * 3 + 0) * L->n + i] = jx;
            j[(s * 3 + 1) * L->n + i] = jy;
            j[(s * 3 + 2) * L->n + i] = jz;
        }
}

/* Eq. FORCE (two belts), the cross repulsion and the body force of every species at every site. */
static void forces(const lbmref3 *L, const double *rho, double *psi, double *F /*[ns][3][n]*/) {
    const double wn = L->p.weight_norm;
    for (int s = 0; s < L->ns; ++s)
        for (long long i = 0; i < L->n; ++i) psi[s * L->n + i] = psi_of(L, s, rho[s * L->n + i]);
    for (int s = 0; s < L->ns; ++s)
#pragma omp parallel for schedule(static)
        for (int z = 0; z < L->nz; ++z)
            for (int y = 0; y < L->ny; ++y)
                for (int x = 0; x < L->nx; ++x) {
                    const long long i = idx(L, x, y, z);
                    double a[3] = {0.0, 0.0, 0.0};
                    for (int k = 0; k < NLINK; ++k) {
                        const int *c = LINKS[k];
                        const int q = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
                        const double K = wn * (L->p.G1[s] * W_ATT[q] + L->p.G2[s] * W_REP[q]);
                        const double pn = psi[s * L->n + nbr(L, x + c[0], y + c[1], z + c[2])];
                        for (int d = 0; d < 3; ++d) a[d] += K * pn * c[d];
                    }
                    double Fs[3];
                    for (int d = 0; d < 3; ++d) Fs[d] = -psi[s * L->n + i] * a[d];
                    if (L->ns == 2) {  /* cross term: species s sees the other's density */
                        const int o = 1 - s;
                        double b[3] = {0.0, 0.0, 0.0};
                        for (int l = 1; l < 19; ++l) {
                            const int *c = C19[l];
                            const int q = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
                            const double rn = rho[o * L->n + nbr(L, x + c[0], y + c[1], z + c[2])];
                            for (int d = 0; d < 3; ++d) b[d] += wn * W_CROSS[q] * rn * c[d];
                        }
                        for (int d = 0; d < 3; ++d) Fs[d] += -L->p.G_AB * rho[s * L->n + i] * b[d];
                    }
                    Fs[0] += rho[s * L->n + i] * L->p.body_force;
                    for (int d = 0; d < 3; ++d) F[(s * 3 + d) * L->n + i] = Fs[d];
                }
}

int lbmref3_site_fields(lbmref3 *L, double *psi_out, double *F_out) {
    if (!L) return 1;
    double *rho = (double *)malloc(sizeof(double) * (size_t)(L->ns * L->n));
    double *j = (double *)malloc(sizeof(double) * (size_t)(L->ns * 3 * L->n));
    double *psi = (double *)malloc(sizeof(double) * (size_t)(L->ns * L->n));
    double *F = (double *)malloc(sizeof(double) * (size_t)(L->ns * 3 * L->n));
    if (!rho || !j || !psi || !F) {
        free(rho);
        free(j);
        free(psi);
        free(F);
        return 3;
    }
    moments(L, rho, j);
    forces(L, rho, psi, F);
    if (psi_out) memcpy(psi_out, psi, sizeof(double) * (size_t)(L->ns * L->n));
    if (F_out) memcpy(F_out, F, sizeof(double) * (size_t)(L->ns * 3 * L->n));
    free(rho);
    free(j);
    free(psi);
    free(F);
    return 0;
}

/* One time step: moments and forces of the current state, shifted-velocity BGK collision of
   Sec. II, then streaming f_l(x + c_l, t + 1) = f*_l(x, t) (periodic). */
static int step1(lbmref3 *L) {
    const long long n = L->n;
    const int ns = L->ns;
    double *rho = (double *)malloc(sizeof(double) * (size_t)(ns * n));
    double *j = (double *)malloc(sizeof(double) * (size_t)(ns * 3 * n));
    double *psi = (double *)malloc(sizeof(double) * (size_t)(ns * n));
    double *F = (double *)malloc(sizeof(double) * (size_t)(ns * 3 * n));
    if (!rho || !j || !psi || !F) {
        free(rho);
        free(j);
        free(psi);
        free(F);
        return 3;
    }
    moments(L, rho, j);
    forces(L, rho, psi, F);
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < n; ++i) {
        /* common velocity u' = sum_s (j_s / tau_s) / sum_s (rho_s / tau_s) */
        double num[3] = {0.0, 0.0, 0.0}, den = 0.0;
        for (int s = 0; s < ns; ++s) {
            for (int d = 0; d < 3; ++d) num[d] += j[(s * 3 + d) * n + i] / L->p.tau[s];
            den += rho[s * n + i] / L->p.tau[s];
        }
        for (int s = 0; s < ns; ++s) {
            const double r = rho[s * n + i], tau = L->p.tau[s];
            double ueq[3];
            for (int d = 0; d < 3; ++d) ueq[d] = num[d] / den + tau * F[(s * 3 + d) * n + i] / r;
            for (int l = 0; l < 19; ++l) {
                const double fl = L->f[(s * 19 + l) * n + i];
                L->f[(s * 19 + l) * n + i] = fl - (fl - feq(l, r, ueq)) / tau;
            }
        }
    }
    for (int s = 0; s < ns; ++s)
        for (int l = 0; l < 19; ++l)
#pragma omp parallel for schedule(static)
            for (int z = 0; z < L->nz; ++z)
                for (int y = 0; y < L->ny; ++y)
                    for (int x = 0; x < L->nx; ++x) {
                        const long long i = idx(L, x, y, z);
                        const int zd = z + C19[l][2];
                        const double v = L->f[(s * 19 + l) * n + i];
                        if (L->p.zbc && (zd < 0 || zd >= L->nz)) {
                            /* halfway bounce-back: back into this site as opp(l), with Ladd's
                               term for a wall moving along x: -6 W_l rho (c_l . U_w) */
                            const double uw = zd < 0 ? L->p.wall_u[0] : L->p.wall_u[1];
                            L->ftmp[(s * 19 + opp19(l)) * n + i] = v - 6.0 * w19(l) * rho[s * n + i] * C19[l][0] * uw;
                        } else {
                            L->ftmp[(s * 19 + l) * n + idx(L, x + C19[l][0], y + C19[l][1], zd)] = v;
                        }
                    }
    double *t = L->f;
    L->f = L->ftmp;
    L->ftmp = t;
    free(rho);
    free(j);
    free(psi);
    free(F);
    L->steps += 1;
    return 0;
}

int lbmref3_step(lbmref3 *L, int nsteps) {
    if (!L || nsteps < 0) return 1;
    for (int k = 0; k < nsteps; ++k) {
        const int rc = step1(L);
        if (rc) return rc;
    }
    return 0;
}

/* rho [ns][nz][ny][nx], u [3][nz][ny][nx] (barycentric: (sum_s j_s + F_s / 2) / sum_s rho_s),
   f [ns][19][nz][ny][nx]; any may be NULL. */
int lbmref3_get(lbmref3 *L, double *rho_out, double *u_out, double *f_out) {
    if (!L) return 1;
    const long long n = L->n;
    const int ns = L->ns;
    double *rho = (double *)malloc(sizeof(double) * (size_t)(ns * n));
    double *j = (double *)malloc(sizeof(double) * (size_t)(ns * 3 * n));
    double *psi = (double *)malloc(sizeof(double) * (size_t)(ns * n));
    double *F = (double *)malloc(sizeof(double) * (size_t)(ns * 3 * n));
    if (!rho || !j || !psi || !F) {
        free(rho);
        free(j);
        free(psi);
        free(F);
        return 3;
    }
    moments(L, rho, j);
    if (rho_out) memcpy(rho_out, rho, sizeof(double) * (size_t)(ns * n));
    if (u_out) {
        forces(L, rho, psi, F);
        for (long long i = 0; i < n; ++i) {
            double m[3] = {0.0, 0.0, 0.0}, rt = 0.0;
            for (int s = 0; s < ns; ++s) {
                for (int d = 0; d < 3; ++d) m[d] += j[(s * 3 + d) * n + i] + 0.5 * F[(s * 3 + d) * n + i];
                rt += rho[s * n + i];
            }
            for (int d = 0; d < 3; ++d) u_out[d * n + i] = m[d] / rt;
        }
    }
    if (f_out) memcpy(f_out, L->f, sizeof(double) * (size_t)(ns * 19 * n));
    free(rho);
    free(j);
    free(psi);
    free(F);
    return 0;
}

long long lbmref3_step_count(const lbmref3 *L) { return L ? L->steps : -1; }
