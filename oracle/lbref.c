/*
 * lbref.c — ORACLE (test infrastructure only; see lbref.h).
 *
 * Plain FP64 CPU restatement of the time step of §2 of Günther et al.,
 * arXiv:1109.3277: the lattice Boltzmann equation (Eq. 1) with the BGK
 * operator (Eq. 2) on D3Q19, the Shan–Chen inter-component force (Eq. 3)
 * entering the collision, moving bounce-back on particle surfaces (Eq. 4) with
 * the momentum-exchange force (Eq. 5), the anisotropic Hertz potential with
 * the Berne–Pechukas ε, σ (Eq. 6–8), the lubrication correction (Eq. 9), the
 * outer-shell density fill and the particle colour Δρ (Eq. 10 and the text
 * after it).  Where the paper is silent the reading used is stated at the
 * function that takes it.
 *
 * Everything runs in plain loops over nodes in x-fastest raster order, one
 * phase after another, exactly in the order of the step below; nothing is
 * fused, blocked or reordered.  Compile with -ffp-contract=off so that no
 * multiply-add is contracted.
 */
#include "lbref.h"
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define Q 19
enum { T_FLUID = 0, T_WALL = 1, T_PART = 2 };

/* D3Q19 (§2, "a D3Q19 implementation"): rest, 6 axis and 12 face-diagonal
 * velocities, weights 1/3, 1/18, 1/36; opposite directions are adjacent. */
static const int CV[Q][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double WV[Q] = {
    1.0 / 3.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int OPPV[Q] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};

typedef struct {
    double X[3], q[4], V[3], W[3];     /* position, orientation, velocity, ω (lab) */
    double rp, ro, drho;               /* radii along / across the axis, colour Δρ */
    double M, Ipar, Iperp;             /* mass, body-frame inertia */
    double Flink[3], Tlink[3];         /* momentum exchange of this step (Eq. 5) */
    double Fpair[3], Tpair[3];         /* Hertz + lubrication of this step */
    double Fpend[3], Tpend[3];         /* fill/empty momentum, applied next step */
    double F[3], T[3];                 /* total force/torque of the last update */
} particle;

struct lbref_ctx {
    lbref_lattice_desc d;
    long N;
    double *f, *fs;                    /* f: post-streaming state; fs: post-collision */
    double *rho, *jm, *psi, *frc;      /* per-step fields: ρ^c, j^c, ψ^c, F^c */
    unsigned char *type;
    int *owner, *nowner;
    int np, cap;
    particle *p;
    double diag[6];
    char err[256];
};

/* ------------------------------------------------------------------ helpers */

static long nidx(const lbref_ctx *c, int x, int y, int z)
{
    return (long)x + (long)c->d.nx * ((long)y + (long)c->d.ny * (long)z);
}

/* Neighbour of node (x,y,z) along c_i: periodic in x and y, periodic in z
 * unless walls are present, in which case leaving [0,nz) means "no node". */
static long neighbour(const lbref_ctx *c, int x, int y, int z, int i)
{
    int xx = x + CV[i][0], yy = y + CV[i][1], zz = z + CV[i][2];
    if (xx < 0) xx += c->d.nx;
    if (xx >= c->d.nx) xx -= c->d.nx;
    if (yy < 0) yy += c->d.ny;
    if (yy >= c->d.ny) yy -= c->d.ny;
    if (c->d.walls_z) {
        if (zz < 0 || zz >= c->d.nz) return -1;
    } else {
        if (zz < 0) zz += c->d.nz;
        if (zz >= c->d.nz) zz -= c->d.nz;
    }
    return nidx(c, xx, yy, zz);
}

static void coords(const lbref_ctx *c, long n, int *x, int *y, int *z)
{
    *x = (int)(n % c->d.nx);
    *y = (int)((n / c->d.nx) % c->d.ny);
    *z = (int)(n / ((long)c->d.nx * c->d.ny));
}

static int periodic_dim(const lbref_ctx *c, int k) { return k < 2 || !c->d.walls_z; }

static int extent(const lbref_ctx *c, int k) { return k == 0 ? c->d.nx : (k == 1 ? c->d.ny : c->d.nz); }

/* Displacement of integer node coordinate xi from a particle coordinate X:
 * nearest periodic image, taken by shifting the integer first and then
 * subtracting once. */
static double node_disp(const lbref_ctx *c, int k, int xi, double X)
{
    if (periodic_dim(c, k)) {
        int n = extent(c, k);
        double s = rint(((double)xi - X) / (double)n);
        return (double)((long)xi - (long)s * n) - X;
    }
    return (double)xi - X;
}

/* Nearest-image difference of two particle coordinates. */
static double pair_disp(const lbref_ctx *c, int k, double a, double b)
{
    double r = b - a;
    if (periodic_dim(c, k)) {
        double n = (double)extent(c, k);
        r = r - n * rint(r / n);
    }
    return r;
}

static void cross(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Rotation matrix of a unit quaternion q = (w, x, y, z): v_lab = R v_body. */
static void rotmat(const double q[4], double R[3][3])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1.0 - 2.0 * (y * y + z * z);
    R[0][1] = 2.0 * (x * y - w * z);
    R[0][2] = 2.0 * (x * z + w * y);
    R[1][0] = 2.0 * (x * y + w * z);
    R[1][1] = 1.0 - 2.0 * (x * x + z * z);
    R[1][2] = 2.0 * (y * z - w * x);
    R[2][0] = 2.0 * (x * z - w * y);
    R[2][1] = 2.0 * (y * z + w * x);
    R[2][2] = 1.0 - 2.0 * (x * x + y * y);
}

static void qmul(const double a[4], const double b[4], double o[4])
{
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

static void qnormalise(double q[4])
{
    double s = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int k = 0; k < 4; k++) q[k] /= s;
}

/* Quadric inside test of a node against an ellipsoid (reading: a node
 * belongs to the particle iff its body-frame quadric value is <= 1). */
static int inside_disp(const double dx[3], const double R[3][3], double rp, double ro)
{
    double d[3];
    for (int k = 0; k < 3; k++) d[k] = R[0][k] * dx[0] + R[1][k] * dx[1] + R[2][k] * dx[2];
    double ip2 = 1.0 / (rp * rp), io2 = 1.0 / (ro * ro);
    double qv = d[0] * d[0] * ip2 + d[1] * d[1] * io2 + d[2] * d[2] * io2;
    return qv <= 1.0;
}

int lbref_inside(const double node[3], const double pos[3], const double quat[4], double r_par,
                 double r_perp)
{
    double R[3][3], dx[3];
    rotmat(quat, R);
    for (int k = 0; k < 3; k++) dx[k] = node[k] - pos[k];
    return inside_disp(dx, R, r_par, r_perp);
}

void lbref_lattice(int32_t *c, double *w, int32_t *opp)
{
    for (int i = 0; i < Q; i++) {
        for (int k = 0; k < 3; k++) c[3 * i + k] = CV[i][k];
        w[i] = WV[i];
        opp[i] = OPPV[i];
    }
}

/* Equilibrium of the BGK operator (Eq. 2).  The paper does not print f^eq;
 * the standard second-order D3Q19 form with c_s^2 = 1/3 is used. */
void lbref_feq(double rho, const double u[3], double *feq)
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; i++) {
        double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
        feq[i] = WV[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

static void seterr(lbref_ctx *c, const char *m)
{
    if (c) snprintf(c->err, sizeof c->err, "%s", m);
}

const char *lbref_last_error(const lbref_ctx *c) { return c ? c->err : "null context"; }

/* ------------------------------------------------------------ construction */

int lbref_init_lattice(const lbref_lattice_desc *d, const double *rho0, lbref_ctx **out)
{
    if (!d || !out || !rho0) return LBREF_EINVAL;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1) return LBREF_EINVAL;
    if (d->walls_z && d->nz < 3) return LBREF_EINVAL;
    if (!(d->tau[0] > 0.5) || !(d->tau[1] > 0.5)) return LBREF_EINVAL;
    lbref_ctx *c = (lbref_ctx *)calloc(1, sizeof *c);
    if (!c) return LBREF_ENOMEM;
    c->d = *d;
    c->N = (long)d->nx * d->ny * d->nz;
    long N = c->N;
    c->f = (double *)calloc((size_t)2 * Q * N, sizeof(double));
    c->fs = (double *)calloc((size_t)2 * Q * N, sizeof(double));
    c->rho = (double *)calloc((size_t)2 * N, sizeof(double));
    c->jm = (double *)calloc((size_t)6 * N, sizeof(double));
    c->psi = (double *)calloc((size_t)2 * N, sizeof(double));
    c->frc = (double *)calloc((size_t)6 * N, sizeof(double));
    c->type = (unsigned char *)calloc((size_t)N, 1);
    c->owner = (int *)malloc((size_t)N * sizeof(int));
    c->nowner = (int *)malloc((size_t)N * sizeof(int));
    if (!c->f || !c->fs || !c->rho || !c->jm || !c->psi || !c->frc || !c->type || !c->owner ||
        !c->nowner) {
        lbref_destroy(c);
        return LBREF_ENOMEM;
    }
    for (long n = 0; n < N; n++) {
        int x, y, z;
        coords(c, n, &x, &y, &z);
        c->owner[n] = -1;
        c->type[n] = (d->walls_z && (z == 0 || z == d->nz - 1)) ? T_WALL : T_FLUID;
        for (int cc = 0; cc < 2; cc++)
            for (int i = 0; i < Q; i++)
                c->f[((long)cc * Q + i) * N + n] =
                    c->type[n] == T_FLUID ? WV[i] * rho0[(long)cc * N + n] : 0.0;
    }
    *out = c;
    return LBREF_OK;
}

void lbref_destroy(lbref_ctx *c)
{
    if (!c) return;
    free(c->f);
    free(c->fs);
    free(c->rho);
    free(c->jm);
    free(c->psi);
    free(c->frc);
    free(c->type);
    free(c->owner);
    free(c->nowner);
    free(c->p);
    free(c);
}

/* Axis-aligned box that contains the ellipsoid, widened by one node.
 * Returns 0 (no box) for non-finite geometry or a centre further than 1e9
 * from the origin; the bounds are formed in double before conversion. */
static int particle_box(const lbref_ctx *c, const particle *P, int lo[3], int hi[3])
{
    double R[3][3];
    rotmat(P->q, R);
    for (int k = 0; k < 3; k++) {
        double h = sqrt(P->rp * P->rp * R[k][0] * R[k][0] +
                        P->ro * P->ro * (R[k][1] * R[k][1] + R[k][2] * R[k][2]));
        double l = floor(P->X[k] - h) - 1.0, u = ceil(P->X[k] + h) + 1.0;
        if (!(l <= u) || !(fabs(P->X[k]) < 1e9) || !(h < 1e9)) return 0;
        int n = extent(c, k);
        if (!periodic_dim(c, k)) {
            if (l < 0) l = 0;
            if (u > n - 1) u = n - 1;
        } else if (u - l + 1 > n) {
            l = 0;
            u = n - 1;
        }
        lo[k] = (int)l;
        hi[k] = (int)u;
    }
    return 1;
}

static int wrapi(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

/* New ownership map: every non-wall node inside a particle belongs to the
 * lowest-indexed particle that contains it. */
static void claim_nodes(lbref_ctx *c, int *own)
{
    for (long n = 0; n < c->N; n++) own[n] = -1;
    for (int p = 0; p < c->np; p++) {
        particle *P = &c->p[p];
        double R[3][3];
        rotmat(P->q, R);
        int lo[3], hi[3];
        if (!particle_box(c, P, lo, hi)) continue;
        for (int z = lo[2]; z <= hi[2]; z++)
            for (int y = lo[1]; y <= hi[1]; y++)
                for (int x = lo[0]; x <= hi[0]; x++) {
                    int xi = wrapi(x, c->d.nx), yi = wrapi(y, c->d.ny), zi = wrapi(z, c->d.nz);
                    long n = nidx(c, xi, yi, zi);
                    if (c->type[n] == T_WALL || own[n] >= 0) continue;
                    double dx[3] = {node_disp(c, 0, xi, P->X[0]), node_disp(c, 1, yi, P->X[1]),
                                    node_disp(c, 2, zi, P->X[2])};
                    if (inside_disp(dx, R, P->rp, P->ro)) own[n] = p;
                }
    }
}

int lbref_add_particles(lbref_ctx *c, int32_t n, const double *pos, const double *quat,
                        const double *vel, const double *omega, const double *r_par,
                        const double *r_perp, const double *delta_rho)
{
    if (!c) return LBREF_EINVAL;
    if (n < 0 || (n > 0 && (!pos || !quat || !r_par || !r_perp || !delta_rho))) {
        seterr(c, "add_particles: bad arguments");
        return LBREF_EINVAL;
    }
    for (int k = 0; k < n; k++) {
        if (!(r_par[k] > 0) || !(r_perp[k] > 0)) {
            seterr(c, "add_particles: radii must be positive");
            return LBREF_EINVAL;
        }
        double qq = quat[4 * k] * quat[4 * k] + quat[4 * k + 1] * quat[4 * k + 1] +
                    quat[4 * k + 2] * quat[4 * k + 2] + quat[4 * k + 3] * quat[4 * k + 3];
        if (!(qq > 0)) {
            seterr(c, "add_particles: zero quaternion");
            return LBREF_EINVAL;
        }
        for (int j = 0; j < 3; j++) {
            double X = pos[3 * k + j];
            if (!(X >= 0) || !(X < extent(c, j))) {
                seterr(c, "add_particles: position outside the lattice");
                return LBREF_EINVAL;
            }
        }
    }
    particle *np = (particle *)realloc(c->p, sizeof(particle) * (size_t)(c->np + n + 1));
    if (!np) return LBREF_ENOMEM;
    c->p = np;
    for (int k = 0; k < n; k++) {
        particle *P = &c->p[c->np + k];
        memset(P, 0, sizeof *P);
        for (int j = 0; j < 3; j++) {
            P->X[j] = pos[3 * k + j];
            P->V[j] = vel ? vel[3 * k + j] : 0.0;
            P->W[j] = omega ? omega[3 * k + j] : 0.0;
        }
        for (int j = 0; j < 4; j++) P->q[j] = quat[4 * k + j];
        qnormalise(P->q);
        P->rp = r_par[k];
        P->ro = r_perp[k];
        P->drho = delta_rho[k];
        /* Reading: particle density 1, solid-ellipsoid inertia about the
         * symmetry axis (0.4 M ro^2) and across it (0.2 M (rp^2 + ro^2)). */
        P->M = (c->d.rho_particle > 0 ? c->d.rho_particle : 1.0) * 4.0 / 3.0 * M_PI * P->rp * P->ro * P->ro;
        P->Ipar = 0.4 * P->M * P->ro * P->ro;
        P->Iperp = 0.2 * P->M * (P->rp * P->rp + P->ro * P->ro);
    }
    c->np += n;
    /* Placement: claim nodes; newly covered nodes lose their fluid (no
     * momentum is transferred at placement). */
    claim_nodes(c, c->nowner);
    for (long m = 0; m < c->N; m++) {
        if (c->type[m] == T_WALL) continue;
        c->owner[m] = c->nowner[m];
        c->type[m] = c->nowner[m] >= 0 ? T_PART : T_FLUID;
        if (c->type[m] == T_PART)
            for (int cc = 0; cc < 2; cc++)
                for (int i = 0; i < Q; i++) c->f[((long)cc * Q + i) * c->N + m] = 0.0;
    }
    return LBREF_OK;
}

/* ------------------------------------------------------------- the step */

/* Phase 1: moments ρ^c = Σ_i f_i^c and j^c = Σ_i f_i^c c_i on fluid nodes (§2). */
static void phase_moments(lbref_ctx *c)
{
    long N = c->N;
#ifdef LBREF_OMP
#pragma omp parallel for schedule(static)
#endif
    for (long n = 0; n < N; n++) {
        for (int cc = 0; cc < 2; cc++) {
            double r = 0, j0 = 0, j1 = 0, j2 = 0;
            if (c->type[n] == T_FLUID) {
                for (int i = 0; i < Q; i++) {
                    double fv = c->f[((long)cc * Q + i) * N + n];
                    r += fv;
                    j0 += fv * CV[i][0];
                    j1 += fv * CV[i][1];
                    j2 += fv * CV[i][2];
                }
            }
            c->rho[cc * N + n] = r;
            c->jm[(cc * 3 + 0) * N + n] = j0;
            c->jm[(cc * 3 + 1) * N + n] = j1;
            c->jm[(cc * 3 + 2) * N + n] = j2;
        }
    }
}

/* Phases 2-3: ψ^c = 1 - exp(-ρ^c) (the monotonous weight of Eq. 3).  On
 * solid nodes with at least one fluid neighbour (the outer shell) ρ^c is
 * first replaced by the mean over those neighbours (Eq. 10) and the colour
 * rule adds Δρ to red if Δρ > 0, else |Δρ| to blue.  Walls take Δρ = 0.
 * Interior solid nodes get ψ = 0; no fluid node ever reads them. */
static void phase_psi(lbref_ctx *c)
{
    long N = c->N;
#ifdef LBREF_OMP
#pragma omp parallel for schedule(static)
#endif
    for (long n = 0; n < N; n++) {
        if (c->type[n] == T_FLUID) {
            for (int cc = 0; cc < 2; cc++) c->psi[cc * N + n] = 1.0 - exp(-c->rho[cc * N + n]);
            continue;
        }
        int x, y, z;
        coords(c, n, &x, &y, &z);
        double s[2] = {0, 0};
        int cnt = 0;
        for (int i = 1; i < Q; i++) {
            long m = neighbour(c, x, y, z, i);
            if (m < 0 || c->type[m] != T_FLUID) continue;
            s[0] += c->rho[m];
            s[1] += c->rho[N + m];
            cnt++;
        }
        if (cnt == 0) {
            c->psi[n] = 0.0;
            c->psi[N + n] = 0.0;
            continue;
        }
        double rn[2] = {s[0] / cnt, s[1] / cnt};
        double dr = c->type[n] == T_PART ? c->p[c->owner[n]].drho : 0.0;
        if (dr > 0)
            rn[0] += dr;
        else
            rn[1] += fabs(dr);
        for (int cc = 0; cc < 2; cc++) c->psi[cc * N + n] = 1.0 - exp(-rn[cc]);
    }
}

/* Phase 4: F^c(x) = -g ψ^c(x) Σ_{i=1..18} ψ^{c'}(x + c_i) c_i on fluid nodes
 * (Eq. 3 with g_rb = g_br = g, g_rr = g_bb = 0; reading: unweighted sum
 * over the 18 neighbours), plus ρ^c times the body force. */
static void phase_force(lbref_ctx *c)
{
    long N = c->N;
    double g = c->d.g_br;
#ifdef LBREF_OMP
#pragma omp parallel for schedule(static)
#endif
    for (long n = 0; n < N; n++) {
        for (int k = 0; k < 6; k++) c->frc[k * N + n] = 0.0;
        if (c->type[n] != T_FLUID) continue;
        int x, y, z;
        coords(c, n, &x, &y, &z);
        for (int cc = 0; cc < 2; cc++) {
            int co = 1 - cc;
            double sx = 0, sy = 0, sz = 0;
            for (int i = 1; i < Q; i++) {
                long m = neighbour(c, x, y, z, i);
                double ps = c->psi[co * N + m];
                sx += ps * CV[i][0];
                sy += ps * CV[i][1];
                sz += ps * CV[i][2];
            }
            double pc = c->psi[cc * N + n], rc = c->rho[cc * N + n];
            c->frc[(cc * 3 + 0) * N + n] = -g * pc * sx + rc * c->d.body_force[0];
            c->frc[(cc * 3 + 1) * N + n] = -g * pc * sy + rc * c->d.body_force[1];
            c->frc[(cc * 3 + 2) * N + n] = -g * pc * sz + rc * c->d.body_force[2];
        }
    }
}

/* Phase 5: BGK collision (Eq. 2) with the force entering through the
 * Shan–Chen shifted velocity: u' = Σ_c (j^c/τ_c) / Σ_c (ρ^c/τ_c), and the
 * equilibrium of component c is taken at u' + τ_c F^c / ρ^c. */
static void phase_collide(lbref_ctx *c)
{
    long N = c->N;
#ifdef LBREF_OMP
#pragma omp parallel for schedule(static)
#endif
    for (long n = 0; n < N; n++) {
        if (c->type[n] != T_FLUID) continue;
        double num[3] = {0, 0, 0}, den = 0;
        for (int cc = 0; cc < 2; cc++) {
            double t = c->d.tau[cc];
            for (int k = 0; k < 3; k++) num[k] += c->jm[(cc * 3 + k) * N + n] / t;
            den += c->rho[cc * N + n] / t;
        }
        double up[3] = {0, 0, 0};
        if (den > 0)
            for (int k = 0; k < 3; k++) up[k] = num[k] / den;
        for (int cc = 0; cc < 2; cc++) {
            double t = c->d.tau[cc], r = c->rho[cc * N + n];
            double ue[3];
            for (int k = 0; k < 3; k++)
                ue[k] = r > 0 ? up[k] + t * c->frc[(cc * 3 + k) * N + n] / r : up[k];
            double feq[Q];
            lbref_feq(r, ue, feq);
            for (int i = 0; i < Q; i++) {
                long a = ((long)cc * Q + i) * N + n;
                c->fs[a] = c->f[a] - (c->f[a] - feq[i]) / t;
            }
        }
    }
}

/* Phase 6: streaming (Eq. 1) by pull; a population that would come from a
 * solid node is the reflected post-collision population of the fluid node
 * itself plus C (Eq. 4), C = 6 w_i ρ^c(y) u_surf·c_i (reading: α = w_i,
 * c_s^2 = 1/3, u_surf at the link midpoint).  Each particle link gives the
 * particle F = (2 f*_ī + C) c_ī (Eq. 5) and the torque r_b × F. */
static void phase_stream(lbref_ctx *c)
{
    long N = c->N;
    double *fn = c->f; /* f is overwritten: fs holds everything needed */
    for (int p = 0; p < c->np; p++)
        for (int k = 0; k < 3; k++) c->p[p].Flink[k] = c->p[p].Tlink[k] = 0.0;
    c->diag[4] = c->diag[5] = 0.0;
    for (long y = 0; y < N; y++) {
        if (c->type[y] != T_FLUID) continue;
        int x0, y0, z0;
        coords(c, y, &x0, &y0, &z0);
        for (int i = 0; i < Q; i++) {
            long src = i == 0 ? y : neighbour(c, x0, y0, z0, OPPV[i]);
            if (src >= 0 && c->type[src] == T_FLUID) {
                for (int cc = 0; cc < 2; cc++)
                    fn[((long)cc * Q + i) * N + y] = c->fs[((long)cc * Q + i) * N + src];
                continue;
            }
            int io = OPPV[i];
            if (src >= 0 && c->type[src] == T_PART) {
                particle *P = &c->p[c->owner[src]];
                double rb[3] = {node_disp(c, 0, x0, P->X[0]) - 0.5 * CV[i][0],
                                node_disp(c, 1, y0, P->X[1]) - 0.5 * CV[i][1],
                                node_disp(c, 2, z0, P->X[2]) - 0.5 * CV[i][2]};
                double wr[3], us[3];
                cross(P->W, rb, wr);
                for (int k = 0; k < 3; k++) us[k] = P->V[k] + wr[k];
                double uc = us[0] * CV[i][0] + us[1] * CV[i][1] + us[2] * CV[i][2];
                for (int cc = 0; cc < 2; cc++) {
                    double fr = c->fs[((long)cc * Q + io) * N + y];
                    double C = 6.0 * WV[i] * c->rho[cc * N + y] * uc;
                    fn[((long)cc * Q + i) * N + y] = fr + C;
                    double F[3], T[3];
                    for (int k = 0; k < 3; k++) F[k] = (2.0 * fr + C) * CV[io][k];
                    cross(rb, F, T);
                    for (int k = 0; k < 3; k++) {
                        P->Flink[k] += F[k];
                        P->Tlink[k] += T[k];
                    }
                    c->diag[4 + cc] += C;
                }
            } else {
                /* wall (or outside the domain): resting halfway bounce-back */
                for (int cc = 0; cc < 2; cc++)
                    fn[((long)cc * Q + i) * N + y] = c->fs[((long)cc * Q + io) * N + y];
            }
        }
    }
}

/* Berne–Pechukas anisotropic Hertz interaction (Eq. 6–8).  Reading:
 * φ̃(s) = (1 - s)^{5/2} for s < 1, ε̄ = K_H σ̄^{5/2}, σ̄ = 2 r_perp, so the
 * sphere limit is K_H (2R - r)^{5/2}.  Force and torques are minus the
 * analytic derivatives with respect to r = X_j - X_i and the two axes. */
void lbref_pair_hertz(double k_hertz, double rp, double ro, const double r[3], const double oi[3],
                      const double oj[3], double *energy, double f_j[3], double t_i[3],
                      double t_j[3], double *sigma_out)
{
    for (int k = 0; k < 3; k++) f_j[k] = t_i[k] = t_j[k] = 0.0;
    *energy = 0.0;
    double chi = (rp * rp - ro * ro) / (rp * rp + ro * ro);
    double sbar = 2.0 * ro;
    double ebar = k_hertz * pow(sbar, 2.5);
    double rl = sqrt(dot(r, r));
    if (!(rl > 0)) {
        *sigma_out = sbar;
        return;
    }
    double rh[3] = {r[0] / rl, r[1] / rl, r[2] / rl};
    double a = dot(rh, oi), b = dot(rh, oj), cc = dot(oi, oj);
    double ep = 1.0 + chi * cc, em = 1.0 - chi * cc;
    double S = (a + b) * (a + b) / ep + (a - b) * (a - b) / em;
    double D = 1.0 - 0.5 * chi * S;
    double sigma = sbar / sqrt(D);
    *sigma_out = sigma;
    double Ed = 1.0 - chi * chi * cc * cc;
    double eps = ebar / sqrt(Ed);
    double s = rl / sigma;
    if (s >= 1.0) return;
    double phit = pow(1.0 - s, 2.5);
    double dphit = -2.5 * pow(1.0 - s, 1.5);
    *energy = eps * phit;
    double dsig_dS = 0.25 * chi * sbar / (D * sqrt(D));
    double dS_da = 2.0 * (a + b) / ep + 2.0 * (a - b) / em;
    double dS_db = 2.0 * (a + b) / ep - 2.0 * (a - b) / em;
    double dS_dc = -chi * (a + b) * (a + b) / (ep * ep) + chi * (a - b) * (a - b) / (em * em);
    double deps_dc = ebar * chi * chi * cc / (Ed * sqrt(Ed));
    double dphi_dsig = eps * dphit * (-rl / (sigma * sigma));
    double dphi_drl = eps * dphit / sigma;
    double gs = dphi_dsig * dsig_dS;
    double grad[3], gi[3], gj[3];
    for (int k = 0; k < 3; k++) {
        grad[k] = dphi_drl * rh[k] + gs * (dS_da * (oi[k] - a * rh[k]) / rl +
                                           dS_db * (oj[k] - b * rh[k]) / rl);
        gi[k] = phit * deps_dc * oj[k] + gs * (dS_da * rh[k] + dS_dc * oj[k]);
        gj[k] = phit * deps_dc * oi[k] + gs * (dS_db * rh[k] + dS_dc * oi[k]);
    }
    for (int k = 0; k < 3; k++) f_j[k] = -grad[k];
    double ti[3], tj[3];
    cross(oi, gi, ti);
    cross(oj, gj, tj);
    for (int k = 0; k < 3; k++) {
        t_i[k] = -ti[k];
        t_j[k] = -tj[k];
    }
}

/* Phase 7a: pair forces.  Hertz/Berne–Pechukas for every pair; the
 * lubrication correction of Eq. 9 with 2R replaced by σ and R^2 by (σ/2)^2,
 * μ = lub_rho ν, ν = (mean τ - 1/2)/3, only for gaps 0 < r - σ < Δc, and
 * signed so that it opposes the normal approach velocity.  Two particles of
 * different shape interact with the mean of their radii.
 *
 * Reading (the paper does not say how its explicit update treats Eq. 9):
 * the coefficient γ = K (1/h - 1/Δc) of the normal relative velocity is
 * capped at the pair's reduced mass M_i M_j / (M_i + M_j).  One update
 * (Δt = 1) changes the normal approach speed by γ/M_red times itself, so at
 * the cap the correction removes the approach in one step; above it the
 * 1/h growth at small gaps would reverse the approach with a larger speed
 * each step and the pair would fly apart. */
static void phase_pairs(lbref_ctx *c)
{
    for (int p = 0; p < c->np; p++)
        for (int k = 0; k < 3; k++) c->p[p].Fpair[k] = c->p[p].Tpair[k] = 0.0;
    double nu = (0.5 * (c->d.tau[0] + c->d.tau[1]) - 0.5) / 3.0;
    double mu = c->d.lub_rho * nu;
    for (int i = 0; i < c->np; i++)
        for (int j = i + 1; j < c->np; j++) {
            particle *A = &c->p[i], *B = &c->p[j];
            double r[3];
            for (int k = 0; k < 3; k++) r[k] = pair_disp(c, k, A->X[k], B->X[k]);
            double RA[3][3], RB[3][3];
            rotmat(A->q, RA);
            rotmat(B->q, RB);
            double oi[3] = {RA[0][0], RA[1][0], RA[2][0]};
            double oj[3] = {RB[0][0], RB[1][0], RB[2][0]};
            double rp = 0.5 * (A->rp + B->rp), ro = 0.5 * (A->ro + B->ro);
            double e, fj[3], ti[3], tj[3], sigma;
            lbref_pair_hertz(c->d.k_hertz, rp, ro, r, oi, oj, &e, fj, ti, tj, &sigma);
            for (int k = 0; k < 3; k++) {
                B->Fpair[k] += fj[k];
                A->Fpair[k] -= fj[k];
                A->Tpair[k] += ti[k];
                B->Tpair[k] += tj[k];
            }
            double rl = sqrt(dot(r, r));
            double h = rl - sigma;
            if (c->d.lub_cut > 0 && h > 0 && h < c->d.lub_cut) {
                double rh[3] = {r[0] / rl, r[1] / rl, r[2] / rl};
                double du[3] = {A->V[0] - B->V[0], A->V[1] - B->V[1], A->V[2] - B->V[2]};
                double K = 3.0 * M_PI * mu * sigma * sigma / 8.0;
                double gam = K * (1.0 / h - 1.0 / c->d.lub_cut);
                double mred = A->M * B->M / (A->M + B->M);
                if (gam > mred) gam = mred;
                double s = gam * dot(rh, du);
                for (int k = 0; k < 3; k++) {
                    A->Fpair[k] -= s * rh[k];
                    B->Fpair[k] += s * rh[k];
                }
            }
        }
}

/* Reading of "Newton's equation in the spirit of classical molecular
 * dynamics": leapfrog for translation (V += F/M, X += V, Δt = 1), explicit
 * Euler for the body-frame Euler equations, then q <- normalise(q ⊗
 * exp(ω_body/2)). */
void lbref_rigid_update(double mass, double i_par, double i_perp, const double force[3],
                        const double torque[3], double *pos, double *quat, double *vel,
                        double *omega)
{
    for (int k = 0; k < 3; k++) {
        vel[k] += force[k] / mass;
        pos[k] += vel[k];
    }
    double R[3][3];
    rotmat(quat, R);
    double wb[3], tb[3];
    for (int k = 0; k < 3; k++) {
        wb[k] = R[0][k] * omega[0] + R[1][k] * omega[1] + R[2][k] * omega[2];
        tb[k] = R[0][k] * torque[0] + R[1][k] * torque[1] + R[2][k] * torque[2];
    }
    double I[3] = {i_par, i_perp, i_perp};
    double L[3] = {I[0] * wb[0], I[1] * wb[1], I[2] * wb[2]};
    double wl[3];
    cross(wb, L, wl);
    for (int k = 0; k < 3; k++) wb[k] += (tb[k] - wl[k]) / I[k];
    double h[3] = {0.5 * wb[0], 0.5 * wb[1], 0.5 * wb[2]};
    double hn = sqrt(dot(h, h));
    double dq[4] = {1.0, 0.0, 0.0, 0.0};
    if (hn > 0) {
        double s = sin(hn) / hn;
        dq[0] = cos(hn);
        dq[1] = s * h[0];
        dq[2] = s * h[1];
        dq[3] = s * h[2];
    }
    double qn[4];
    qmul(quat, dq, qn);
    qnormalise(qn);
    for (int k = 0; k < 4; k++) quat[k] = qn[k];
    rotmat(quat, R);
    for (int k = 0; k < 3; k++) omega[k] = R[k][0] * wb[0] + R[k][1] * wb[1] + R[k][2] * wb[2];
}

static void wrap_position(const lbref_ctx *c, double X[3])
{
    for (int k = 0; k < 3; k++) {
        if (!periodic_dim(c, k)) continue;
        double n = (double)extent(c, k);
        if (X[k] < 0) X[k] += n;
        if (X[k] >= n) X[k] -= n;
    }
}

/* Phase 7b: move the particles with the total force of this step: momentum
 * exchange + pair forces + the fill/empty momentum of the previous step. */
static void phase_integrate(lbref_ctx *c)
{
    for (int p = 0; p < c->np; p++) {
        particle *P = &c->p[p];
        for (int k = 0; k < 3; k++) {
            P->F[k] = P->Flink[k] + P->Fpair[k] + P->Fpend[k];
            P->T[k] = P->Tlink[k] + P->Tpair[k] + P->Tpend[k];
            P->Fpend[k] = P->Tpend[k] = 0.0;
        }
        if (c->d.particle_mode == 1) continue;
        if (c->d.particle_mode == 2) {
            double V[3] = {P->V[0], P->V[1], P->V[2]};
            double W[3] = {P->W[0], P->W[1], P->W[2]};
            /* prescribed motion: same kinematics with no force and no
             * gyroscopic term (ω held fixed in the lab frame) */
            for (int k = 0; k < 3; k++) P->X[k] += V[k];
            double R[3][3];
            rotmat(P->q, R);
            double wb[3];
            for (int k = 0; k < 3; k++) wb[k] = R[0][k] * W[0] + R[1][k] * W[1] + R[2][k] * W[2];
            double h[3] = {0.5 * wb[0], 0.5 * wb[1], 0.5 * wb[2]};
            double hn = sqrt(dot(h, h));
            double dq[4] = {1.0, 0.0, 0.0, 0.0};
            if (hn > 0) {
                double s = sin(hn) / hn;
                dq[0] = cos(hn);
                dq[1] = s * h[0];
                dq[2] = s * h[1];
                dq[3] = s * h[2];
            }
            double qn[4];
            qmul(P->q, dq, qn);
            qnormalise(qn);
            for (int k = 0; k < 4; k++) P->q[k] = qn[k];
        } else {
            lbref_rigid_update(P->M, P->Ipar, P->Iperp, P->F, P->T, P->X, P->q, P->V, P->W);
        }
        wrap_position(c, P->X);
    }
}

/* Phase 8: coverage update with fill and empty (reading of the rule the
 * paper takes from its ref. [Jansen2011]).  A newly covered node loses its
 * fluid; its mass and momentum go to the covering particle.  A newly
 * uncovered node gets f^eq(ρ̄^c, u_surf) with ρ̄^c the mean over neighbours
 * that are fluid before and after the update (rho_ref if none); the
 * particle loses that momentum.  Momentum moves through the pending
 * force/torque that enters the next update. */
static void phase_coverage(lbref_ctx *c)
{
    long N = c->N;
    c->diag[0] = c->diag[1] = c->diag[2] = c->diag[3] = 0.0;
    if (c->np == 0) return;
    claim_nodes(c, c->nowner);
    for (long n = 0; n < N; n++) {
        if (c->type[n] == T_WALL) continue;
        int was = c->type[n] == T_PART, oldp = c->owner[n], newp = c->nowner[n];
        int x, y, z;
        coords(c, n, &x, &y, &z);
        if (!was && newp >= 0) {
            particle *P = &c->p[newp];
            double mom[3] = {0, 0, 0};
            for (int cc = 0; cc < 2; cc++)
                for (int i = 0; i < Q; i++) {
                    double fv = c->f[((long)cc * Q + i) * N + n];
                    c->diag[2 + cc] += fv;
                    for (int k = 0; k < 3; k++) mom[k] += fv * CV[i][k];
                }
            double r[3] = {node_disp(c, 0, x, P->X[0]), node_disp(c, 1, y, P->X[1]),
                           node_disp(c, 2, z, P->X[2])};
            double t[3];
            cross(r, mom, t);
            for (int k = 0; k < 3; k++) {
                P->Fpend[k] += mom[k];
                P->Tpend[k] += t[k];
            }
        } else if (was && newp < 0) {
            particle *P = &c->p[oldp];
            double sr[2] = {0, 0};
            int cnt = 0;
            for (int i = 1; i < Q; i++) {
                long m = neighbour(c, x, y, z, i);
                if (m < 0 || c->type[m] != T_FLUID || c->nowner[m] >= 0) continue;
                for (int cc = 0; cc < 2; cc++)
                    for (int j = 0; j < Q; j++) sr[cc] += c->f[((long)cc * Q + j) * N + m];
                cnt++;
            }
            double rb[2];
            for (int cc = 0; cc < 2; cc++) rb[cc] = cnt > 0 ? sr[cc] / cnt : c->d.rho_ref[cc];
            double r[3] = {node_disp(c, 0, x, P->X[0]), node_disp(c, 1, y, P->X[1]),
                           node_disp(c, 2, z, P->X[2])};
            double wr[3], us[3];
            cross(P->W, r, wr);
            for (int k = 0; k < 3; k++) us[k] = P->V[k] + wr[k];
            double mom[3] = {0, 0, 0};
            for (int cc = 0; cc < 2; cc++) {
                double feq[Q];
                lbref_feq(rb[cc], us, feq);
                for (int i = 0; i < Q; i++) {
                    c->f[((long)cc * Q + i) * N + n] = feq[i];
                    c->diag[cc] += feq[i];
                    for (int k = 0; k < 3; k++) mom[k] += feq[i] * CV[i][k];
                }
            }
            double t[3];
            cross(r, mom, t);
            for (int k = 0; k < 3; k++) {
                P->Fpend[k] -= mom[k];
                P->Tpend[k] -= t[k];
            }
        }
    }
    for (long n = 0; n < N; n++) {
        if (c->type[n] == T_WALL) continue;
        c->owner[n] = c->nowner[n];
        c->type[n] = c->nowner[n] >= 0 ? T_PART : T_FLUID;
    }
}

int lbref_step(lbref_ctx *c, int32_t nsteps)
{
    if (!c || nsteps < 0) return LBREF_EINVAL;
    for (int s = 0; s < nsteps; s++) {
        phase_moments(c);
        phase_psi(c);
        phase_force(c);
        phase_collide(c);
        phase_stream(c);
        phase_pairs(c);
        phase_integrate(c);
        phase_coverage(c);
    }
    return LBREF_OK;
}

/* ------------------------------------------------------------- readers */

int lbref_read_fields(lbref_ctx *c, double *rho, double *vel, uint8_t *node_type)
{
    if (!c) return LBREF_EINVAL;
    long N = c->N;
    phase_moments(c);
    phase_psi(c);
    phase_force(c);
    for (long n = 0; n < N; n++) {
        int fl = c->type[n] == T_FLUID;
        if (rho) {
            rho[n] = fl ? c->rho[n] : 0.0;
            rho[N + n] = fl ? c->rho[N + n] : 0.0;
        }
        if (vel) {
            double tot = c->rho[n] + c->rho[N + n];
            for (int k = 0; k < 3; k++) {
                double m = c->jm[k * N + n] + c->jm[(3 + k) * N + n] +
                           0.5 * (c->frc[k * N + n] + c->frc[(3 + k) * N + n]);
                vel[(long)k * N + n] = (fl && tot > 0) ? m / tot : 0.0;
            }
        }
        if (node_type) node_type[n] = c->type[n];
    }
    return LBREF_OK;
}

int lbref_read_particles(lbref_ctx *c, double *pos, double *quat, double *vel, double *omega,
                         double *force, double *torque)
{
    if (!c) return LBREF_EINVAL;
    for (int p = 0; p < c->np; p++) {
        particle *P = &c->p[p];
        for (int k = 0; k < 3; k++) {
            if (pos) pos[3 * p + k] = P->X[k];
            if (vel) vel[3 * p + k] = P->V[k];
            if (omega) omega[3 * p + k] = P->W[k];
            if (force) force[3 * p + k] = P->F[k];
            if (torque) torque[3 * p + k] = P->T[k];
        }
        if (quat)
            for (int k = 0; k < 4; k++) quat[4 * p + k] = P->q[k];
    }
    return LBREF_OK;
}

int lbref_mass(lbref_ctx *c, double out[2])
{
    if (!c || !out) return LBREF_EINVAL;
    long N = c->N;
    out[0] = out[1] = 0.0;
    for (int cc = 0; cc < 2; cc++)
        for (long n = 0; n < N; n++) {
            if (c->type[n] != T_FLUID) continue;
            for (int i = 0; i < Q; i++) out[cc] += c->f[((long)cc * Q + i) * N + n];
        }
    return LBREF_OK;
}

int lbref_get_populations(lbref_ctx *c, double *f)
{
    if (!c || !f) return LBREF_EINVAL;
    memcpy(f, c->f, sizeof(double) * 2 * Q * (size_t)c->N);
    return LBREF_OK;
}

int lbref_set_populations(lbref_ctx *c, const double *f)
{
    if (!c || !f) return LBREF_EINVAL;
    memcpy(c->f, f, sizeof(double) * 2 * Q * (size_t)c->N);
    return LBREF_OK;
}

int lbref_diagnostics(lbref_ctx *c, double out[6])
{
    if (!c || !out) return LBREF_EINVAL;
    for (int k = 0; k < 6; k++) out[k] = c->diag[k];
    return LBREF_OK;
}

int lbref_momentum(lbref_ctx *c, double out[9])
{
    if (!c || !out) return LBREF_EINVAL;
    long N = c->N;
    for (int k = 0; k < 9; k++) out[k] = 0.0;
    for (long n = 0; n < N; n++) {
        if (c->type[n] != T_FLUID) continue;
        for (int cc = 0; cc < 2; cc++)
            for (int i = 0; i < Q; i++) {
                double fv = c->f[((long)cc * Q + i) * N + n];
                for (int k = 0; k < 3; k++) out[k] += fv * CV[i][k];
            }
    }
    for (int p = 0; p < c->np; p++)
        for (int k = 0; k < 3; k++) {
            out[3 + k] += c->p[p].M * c->p[p].V[k];
            out[6 + k] += c->p[p].Fpend[k];
        }
    return LBREF_OK;
}
