/*
 * lbref — the ORACLE: a plain, slow, FP64 CPU implementation of one time step
 * of the two-component Shan–Chen D3Q19 BGK lattice Boltzmann fluid coupled to
 * rigid ellipsoids (Günther, Janoschek, Frijters, Harting, arXiv:1109.3277, §2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library (include/lbe.h); the two only
 * agree on the interface shape.  Every function is a direct transcription of
 * the passage it cites, with plain loops and no blocking or fusion.
 *
 * Interface: the same calls as the CUDA library, prefixed lbref_.
 * Layout: node index n = x + nx*(y + ny*z); populations f[c][i][n].
 * Component 0 is "red", component 1 is "blue" (§4: the two immiscible fluids).
 */
#ifndef LBREF_H
#define LBREF_H
#include <stdint.h>
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbref_ctx lbref_ctx;

/* Status codes (same values as the CUDA library's). */
enum { LBREF_OK = 0, LBREF_EINVAL = -1, LBREF_ENOMEM = -2, LBREF_ENUMERIC = -4 };

/* Lattice descriptor.  Field meaning matches the CUDA library's descriptor. */
typedef struct {
    int32_t nx, ny, nz;        /* lattice extent */
    int32_t walls_z;           /* 1: one-node walls at z=0 and z=nz-1 (§4 adsorption box) */
    double  tau[2];            /* BGK relaxation time per component (Eq. 2) */
    double  g_br;              /* Shan–Chen coupling g_br > 0 (Eq. 3, §4 values 0.1 / 0.08) */
    double  body_force[3];     /* extra force per unit density (Poiseuille checks) */
    double  rho_ref[2];        /* offset base for 16-bit storage; also the fill density
                                  for a node uncovered with no fluid neighbour */
    int32_t storage;           /* ignored by the oracle: it always computes in FP64 */
    int32_t particle_mode;     /* 0 free Newton–Euler, 1 static, 2 prescribed velocity */
    double  k_hertz;           /* K_H of the Hertz potential (§2: 100) */
    double  lub_cut;           /* Δc of the lubrication correction (§2: 2/3); 0 disables */
    double  lub_rho;           /* density in μ = ν ρ for the lubrication correction */
    void   *cuda_stream;       /* unused by the oracle */
    int32_t device;            /* unused by the oracle */
    int32_t flags;             /* unused by the oracle */
    double  rho_particle;      /* particle mass density (0 means 1): mass ρ_p times volume */
} lbref_lattice_desc;

/* Create a lattice with populations at rest-equilibrium f_i = w_i rho0 (Eq. 2
 * with u = 0).  rho0 is [2][nz][ny][nx]; values on wall nodes are ignored. */
int  lbref_init_lattice(const lbref_lattice_desc *d, const double *rho0, lbref_ctx **out);
/* Add n ellipsoids (symmetry axis = body x axis, radii r_par along it and
 * r_perp across it).  Nodes inside are made solid; their fluid is discarded. */
int  lbref_add_particles(lbref_ctx *c, int32_t n, const double *pos, const double *quat,
                         const double *vel, const double *omega, const double *r_par,
                         const double *r_perp, const double *delta_rho);
int  lbref_step(lbref_ctx *c, int32_t nsteps);
/* rho [2][N] (0 on solid nodes), vel [3][N] = (sum_c j^c + F/2)/rho (0 on solid),
 * node_type [N] (0 fluid, 1 wall, 2 particle).  Any may be NULL. */
int  lbref_read_fields(lbref_ctx *c, double *rho, double *vel, uint8_t *node_type);
int  lbref_read_particles(lbref_ctx *c, double *pos, double *quat, double *vel,
                          double *omega, double *force, double *torque);
int  lbref_mass(lbref_ctx *c, double out[2]);
/* Raw populations f[2][19][N] (post-streaming state). */
int  lbref_get_populations(lbref_ctx *c, double *f);
int  lbref_set_populations(lbref_ctx *c, const double *f);
/* Per-component bookkeeping of the last step: out[0..1] mass created by
 * uncovering, out[2..3] mass deleted by covering, out[4..5] sum of the
 * moving-bounce-back terms C over all links. */
int  lbref_diagnostics(lbref_ctx *c, double out[6]);
/* Total momentum: out[0..2] fluid (sum f c over fluid nodes), out[3..5]
 * particles (sum M V), out[6..8] pending fill/empty momentum not yet applied. */
int  lbref_momentum(lbref_ctx *c, double out[9]);
const char *lbref_last_error(const lbref_ctx *c);
void lbref_destroy(lbref_ctx *c);

/* ---- pieces exposed for the oracle's own pins ---- */
/* D3Q19 velocity table c[19][3] and weights w[19]. */
void lbref_lattice(int32_t *c, double *w, int32_t *opp);
/* Second-order equilibrium f^eq_i(rho, u), i = 0..18. */
void lbref_feq(double rho, const double u[3], double *feq);
/* Anisotropic Hertz pair interaction of §2 (Eq. 5 with the Berne–Pechukas
 * ε and σ): energy, force on j (= -force on i), torques on i and j, for
 * separation r = X_j - X_i and orientations oi, oj (unit body axes). */
void lbref_pair_hertz(double k_hertz, double r_par, double r_perp, const double r[3],
                      const double oi[3], const double oj[3], double *energy,
                      double f_j[3], double t_i[3], double t_j[3], double *sigma);
/* One rigid-body update (the oracle's Newton–Euler scheme) of a single
 * particle under external force/torque; state = pos[3], quat[4], vel[3],
 * omega[3] (lab frame), updated in place. */
void lbref_rigid_update(double mass, double i_par, double i_perp, const double force[3],
                        const double torque[3], double *pos, double *quat, double *vel,
                        double *omega);
/* Inside test for node coordinates (unwrapped) against one ellipsoid. */
int  lbref_inside(const double node[3], const double pos[3], const double quat[4],
                  double r_par, double r_perp);

#ifdef __cplusplus
}
#endif
#endif
